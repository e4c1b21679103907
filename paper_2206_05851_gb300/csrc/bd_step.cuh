// The step of Eq. 1 on a lane's bonds, shared by every kernel that
// integrates a slot: launch-bound defaults, the per-chain step constants,
// the lane's place in its slot, the step itself and the bond loads/stores.
// (The layout and the arithmetic conventions are described in bd_window.cuh.)
#pragma once

#include "bd_device.cuh"

namespace bdra {

// Launch bound per tile: float 512 threads (16 warps, 128 registers: four
// warps on each SM sub-partition), double 256 threads. The build may override
// them (BD_F32_THREADS / BD_F32_MIN_BLOCKS) to trade registers for warps.
#ifndef BD_F32_THREADS
#define BD_F32_THREADS 512
#endif
#ifndef BD_F32_MIN_BLOCKS
#define BD_F32_MIN_BLOCKS 1
#endif
#ifndef BD_F64_THREADS
#define BD_F64_THREADS 256
#endif
template <typename T, int L> struct Tile {
    static constexpr int max_threads = (sizeof(T) == 4) ? BD_F32_THREADS : BD_F64_THREADS;
    static constexpr int min_blocks = (sizeof(T) == 4) ? BD_F32_MIN_BLOCKS : 1;
};

template <typename T> __device__ __forceinline__ T shfl(T v, int src)
{
    return __shfl_sync(0xffffffffu, v, src);
}

// Per-chain constants of the step, in the integration precision. The noise
// coefficient carries the sign convention of the normals (Normals::sign).
template <typename T, bool FAST> struct StepConst {
    T H, Hinvb, smin;
    T cd;                  // D dt
    T cn;                  // sqrt(2 D dt), times the sign convention of the normals
    T axx, ayy, azz, axz;  // kappa dt
    __device__ __forceinline__ void load(const ChainDev& ch, const StepParams& p)
    {
        if (sizeof(T) == 4 && FAST) {
            // host-rounded float constants (ChainDev::f32)
            H = (T)ch.f32[0]; Hinvb = (T)ch.f32[1]; cd = (T)ch.f32[2]; cn = (T)ch.f32[3];
            axx = (T)ch.f32[4]; ayy = (T)ch.f32[5]; azz = (T)ch.f32[6]; axz = (T)ch.f32[7];
            smin = (T)ch.f32[8];
        } else {
            H = (T)ch.H; Hinvb = (T)ch.Hinvb; smin = (T)p.s_min;
            cd = (T)(0.25 * p.dt);
            cn = (T)sqrt(0.5 * p.dt) * (T)Normals<T, FAST>::sign;
            axx = (T)(ch.kxx * p.dt); ayy = (T)(ch.kyy * p.dt);
            azz = (T)(ch.kzz * p.dt); axz = (T)(ch.kxz * p.dt);
        }
    }
};

// Per-lane position inside its slot.
struct LaneCtx {
    int bead0, nb;
    int nv;                // springs of this lane inside the chain (0 if inactive)
    int src_prev, src_next;
    bool has_prev, has_next, active;
    uint32_t slot_key, chain;
    uint32_t noise_word, noise_half;   // counter word 1 and half of the slot's normals
};

__device__ __forceinline__ LaneCtx make_lane(int seg, int G, int L, int lane, int nb, bool active,
                                             uint32_t slot_key, uint32_t chain)
{
    LaneCtx c;
    c.bead0 = seg * L;
    c.nb = nb;
    c.nv = active ? max(0, min(L, nb - seg * L)) : 0;
    c.has_prev = seg > 0;
    c.has_next = seg + 1 < G;
    c.src_prev = c.has_prev ? lane - 1 : lane;
    c.src_next = c.has_next ? lane + 1 : lane;
    c.active = active;
    c.slot_key = slot_key;
    c.chain = chain;
    c.noise_word = noise_word(slot_key);
    c.noise_half = noise_half(slot_key);
    return c;
}

// One Eq. 1 step of the lane's L bonds; every lane of the warp must call it.
// Returns how many spring forces hit the FENE floor. With TAB the noise comes
// from the split generator: ptab[b] holds PhiloxSplit::bead_part of the
// lane's bead b (indexed from the lane's slot), the step part is computed
// here once per step. H: the slot's noise half when the caller knows it at
// compile time (every lane of the warp the same), -1 to read lc.noise_half.
template <typename T, int L, bool FAST, bool TAB = false, int H = -1>
__device__ __forceinline__ int step_bonds(T (&qx)[L], T (&qy)[L], T (&qz)[L], const LaneCtx& lc,
                                          const StepConst<T, FAST>& k, uint32_t step,
                                          const StepParams& p, const uint4* ptab = nullptr)
{
    int fl = 0;
    uint3 sp = make_uint3(0u, 0u, 0u);
    if (TAB) sp = PhiloxSplit::step_part(step, lc.noise_word, p.rk0);
    const T c0 = spring_coef<T, FAST>(qx[0], qy[0], qz[0], k.H, k.Hinvb, k.smin, fl);
    const T f0x = c0 * qx[0], f0y = c0 * qy[0], f0z = c0 * qz[0];
    T fLx = f0x, fLy = f0y, fLz = f0z;
    if (L > 1) {
        const T cL = spring_coef<T, FAST>(qx[L - 1], qy[L - 1], qz[L - 1], k.H, k.Hinvb, k.smin, fl);
        fLx = cL * qx[L - 1]; fLy = cL * qy[L - 1]; fLz = cL * qz[L - 1];
    }
    // halo springs: the last one of the previous lane, the first of the next
    T fmx = shfl(fLx, lc.src_prev), fmy = shfl(fLy, lc.src_prev), fmz = shfl(fLz, lc.src_prev);
    T fnx = shfl(f0x, lc.src_next), fny = shfl(f0y, lc.src_next), fnz = shfl(f0z, lc.src_next);
    if (!lc.has_prev) { fmx = T(0); fmy = T(0); fmz = T(0); }
    if (!lc.has_next) { fnx = T(0); fny = T(0); fnz = T(0); }
    // noise of this lane's first bead; the next lane's first bead closes our last spring
    T xcx, xcy, xcz;
    if (TAB)
        bead_noise_split<T, FAST, H>(ptab[lc.bead0], sp, p, lc.noise_half, xcx, xcy, xcz);
    else
        bead_noise<T, FAST, H>((uint32_t)lc.bead0, lc.slot_key, step, lc.chain, p, xcx, xcy, xcz);
    const T hx = shfl(xcx, lc.src_next), hy = shfl(xcy, lc.src_next), hz = shfl(xcz, lc.src_next);

    T fcx = f0x, fcy = f0y, fcz = f0z;
#pragma unroll
    for (int j = 0; j < L; ++j) {
        T fpx, fpy, fpz, xnx, xny, xnz;
        if (j + 1 < L) {
            if (j + 1 == L - 1) {
                fpx = fLx; fpy = fLy; fpz = fLz;
            } else {
                const T c = spring_coef<T, FAST>(qx[j + 1], qy[j + 1], qz[j + 1], k.H, k.Hinvb,
                                                 k.smin, fl);
                fpx = c * qx[j + 1]; fpy = c * qy[j + 1]; fpz = c * qz[j + 1];
            }
            if (TAB) {
                uint32_t bj = (uint32_t)(lc.bead0 + j + 1);
                asm volatile("" : "+r"(bj));     // keep the table load inside the step loop
                bead_noise_split<T, FAST, H>(ptab[bj], sp, p, lc.noise_half, xnx, xny, xnz);
            } else {
                bead_noise<T, FAST, H>((uint32_t)(lc.bead0 + j + 1), lc.slot_key, step, lc.chain, p,
                                    xnx, xny, xnz);
            }
        } else {
            fpx = fnx; fpy = fny; fpz = fnz;
            xnx = hx; xny = hy; xnz = hz;
        }
        if (j < lc.nv) {
            const T lx = fma(T(-2), fcx, fpx + fmx);
            const T ly = fma(T(-2), fcy, fpy + fmy);
            const T lz = fma(T(-2), fcz, fpz + fmz);
            const T ox = qx[j], oy = qy[j], oz = qz[j];
            qx[j] = fma(k.cn, xnx - xcx, fma(k.cd, lx, fma(k.axz, oz, fma(k.axx, ox, ox))));
            qy[j] = fma(k.cn, xny - xcy, fma(k.cd, ly, fma(k.ayy, oy, oy)));
            qz[j] = fma(k.cn, xnz - xcz, fma(k.cd, lz, fma(k.azz, oz, oz)));
        }
        fmx = fcx; fmy = fcy; fmz = fcz;
        fcx = fpx; fcy = fpy; fcz = fpz;
        xcx = xnx; xcy = xny; xcz = xnz;
    }
    return lc.active ? fl : 0;
}

template <typename T, int L>
__device__ __forceinline__ void load_bonds(T (&qx)[L], T (&qy)[L], T (&qz)[L], const T* src,
                                           const LaneCtx& lc)
{
#pragma unroll
    for (int j = 0; j < L; ++j) {
        const int i = lc.bead0 + j;
        if (lc.active && i < lc.nb) {
            qx[j] = src[3 * i + 0]; qy[j] = src[3 * i + 1]; qz[j] = src[3 * i + 2];
        } else {
            qx[j] = T(0); qy[j] = T(0); qz[j] = T(0);
        }
    }
}

template <typename T, int L>
__device__ __forceinline__ void store_bonds(const T (&qx)[L], const T (&qy)[L], const T (&qz)[L],
                                            T* dst, const LaneCtx& lc)
{
#pragma unroll
    for (int j = 0; j < L; ++j) {
        const int i = lc.bead0 + j;
        if (lc.active && i < lc.nb) {
            dst[3 * i + 0] = qx[j]; dst[3 * i + 1] = qy[j]; dst[3 * i + 2] = qz[j];
        }
    }
}

}  // namespace bdra
