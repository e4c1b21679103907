// The hot kernels of replica-averaged Brownian dynamics (Sec. II).
//
// Layout. A slot (a parent or one replica) is a run of G = ceil(N / L)
// consecutive lanes of one warp; lane `seg` of the run owns beads and springs
// seg*L .. seg*L + L-1 and keeps those L bond vectors in registers for the
// whole launch. A warp holds P = floor(32 / G) slots. Springs on the
// neighbouring lanes are reached with warp shuffles, so a step touches neither
// shared nor global memory.
//
// Two kernels share one step routine:
//   parent_kernel  advances every parent, writes its conformation at each
//                  window start (the "halted parent" that replicas copy), and
//                  samples it every step (ISF criteria, TSF sums);
//   replica_kernel one CTA per (chain, replica group) evolves the replicas
//                  window after window: spawn from the parent snapshot, S
//                  steps, one force sample per replica at the window end,
//                  float64 cross-replica sum.
// The parent never reads replica state, so integrating it ahead of its
// replicas leaves every result unchanged; the noise is keyed by
// (bead, slot, step, chain), not by launch order.
//
// Bond form of Eq. 1. With free draining (Eq. 2) the update of bead i is
//   r_i += [kappa r_i + D (F_i - F_{i-1})] dt + sqrt(2 D dt) xi_i, D = 1/4,
// so the bond Q_i = r_{i+1} - r_i obeys, exactly,
//   Q_i += [kappa Q_i + D (F_{i+1} - 2 F_i + F_{i-1})] dt
//          + sqrt(2 D dt) (xi_{i+1} - xi_i),
// with F_{-1} = F_{N-1} = 0. The centre of mass, on which no force acts in a
// free-draining chain, is not carried: positions are reported in the
// centre-of-mass frame, and float32 bonds keep full relative precision however
// far a chain drifts or stretches.
//
// These units are compiled with -fmad=false: every fused multiply-add is an
// explicit fma(), so the arithmetic of a step is the same sequence of
// roundings in both kernels and for every tile size L.
#pragma once

#include "bd_conf.cuh"
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
    return c;
}

// One Eq. 1 step of the lane's L bonds; every lane of the warp must call it.
// Returns how many spring forces hit the FENE floor. With TAB the noise comes
// from the split generator: ptab[b] holds PhiloxSplit::bead_part of the
// lane's bead b (indexed from the lane's slot), the step part is computed
// here once per step.
template <typename T, int L, bool FAST, bool TAB = false>
__device__ __forceinline__ int step_bonds(T (&qx)[L], T (&qy)[L], T (&qz)[L], const LaneCtx& lc,
                                          const StepConst<T, FAST>& k, uint32_t step,
                                          const StepParams& p, const uint4* ptab = nullptr)
{
    int fl = 0;
    uint3 sp = make_uint3(0u, 0u, 0u);
    if (TAB) sp = PhiloxSplit::step_part(step, lc.slot_key | ((uint32_t)STREAM_BD << 24), p.rk0);
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
        bead_noise_split<T, FAST>(ptab[lc.bead0], sp, p, xcx, xcy, xcz);
    else
        bead_noise<T, FAST>((uint32_t)lc.bead0, lc.slot_key, step, lc.chain, p, xcx, xcy, xcz);
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
                bead_noise_split<T, FAST>(ptab[bj], sp, p, xnx, xny, xnz);
            } else {
                bead_noise<T, FAST>((uint32_t)(lc.bead0 + j + 1), lc.slot_key, step, lc.chain, p,
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

// ---------------------------------------------------------------------------
// Replicas, one warp work item (one replica per lane run). Lane run s of the
// warp is replica rep_begin + s + 1; state of replica k lives at
// state[(state_off + k (N-1)) * 3 ...]. Snapshots: snap[((w % win_ring) * M +
// spr_off + i) * 3 + d], written by the parent kernel at every window start
// of the current chunk. wsm: this warp's scratch of kWarpScratch values.
// ---------------------------------------------------------------------------
constexpr int kWarpScratch = 512;   // >= slots per warp x springs = P (N-1) <= 32 L

// Eq. 5 diagnostics of a work item's replicas (one per lane run) at the end
// of window w; their bonds were just stored at state_slot (slot base of the
// lane's replica).
template <typename T, int L>
__device__ __noinline__ void conformation_item(const ItemDev& it, const ChainDev& ch,
                                               const StepParams& p, int w, const T* state_slot,
                                               int sw, int P, int G, int bead0, bool active,
                                               int kglob)
{
    const SlotRun r = slot_run((int)(threadIdx.x & 31), sw, P, G);
    const T* pc = reinterpret_cast<const T*>(p.snap) + ((int64_t)(w % p.win_ring) * p.M + ch.spr_off) * 3;
    T acc[L][3];
#pragma unroll
    for (int j = 0; j < L; ++j) acc[j][0] = acc[j][1] = acc[j][2] = T(0);
    eq5_replica<T, L>(state_slot, pc, bead0, r, ch.N, active, acc,
                      p.dbar + ((int64_t)w * p.n_rep + ch.rep_off + kglob - 1) * 3);
    if (it.group == 0)
        eq5_rgz<T, L>(pc, bead0, r, ch.N, sw == 0, p.rgz + (int64_t)w * p.n_chains + it.chain);
    eq5_beads_out<T, L>(acc, bead0, r, sw, P, ch.N, it.rep_count,
                     p.dbead_part + ((int64_t)(w % p.win_ring) * p.bpart_stride + ch.bpart_off +
                                     (int64_t)it.group * ch.N) * 3);
}

// Window end: float64 sum over this warp's replicas of each spring's force,
// in replica order, one partial per (window, spring, group).
template <typename T>
__device__ __forceinline__ void warp_window_sum(const T* wsm, int nb, int count, double* prow)
{
    __syncwarp();
    for (int i = (int)(threadIdx.x & 31); i < nb; i += 32) {
        double acc = 0.0;
        for (int s = 0; s < count; ++s) acc += (double)wsm[s * nb + i];
        prow[i] = acc;
    }
    __syncwarp();
}

// With TAB, ptab is this warp's table of 32 L bead parts of the Philox
// counter (filled here for the item's chain). CONF compiles in the Eq. 5
// window-end diagnostics (used when BD_FLAG_CONFORMATION is set); without it
// the step loop carries no trace of them.
template <typename T, int L, bool FAST, bool TAB = false, bool CONF = false>
__device__ __forceinline__ void run_one_item(const ItemDev& it, const StepParams& p, T* wsm,
                                             uint4* ptab = nullptr)
{
    const ChainDev ch = p.chains[it.chain];
    const int nb = ch.N - 1;
    const int G = (ch.N + L - 1) / L;
    const int P = 32 / G;
    const int lane = threadIdx.x & 31;
    const int sw = lane / G;
    const bool active = (sw < P) && (sw < it.rep_count);
    const int kglob = it.rep_begin + sw + 1;
    const uint32_t key = (p.flags & BD_FLAG_IDENTICAL_NOISE) ? 0u : (uint32_t)kglob;
    const LaneCtx lc = make_lane(sw < P ? lane - sw * G : 0, G, L, lane, nb, active, key,
                                 (uint32_t)it.chain);
    StepConst<T, FAST> k;
    k.load(ch, p);
    if (TAB) {
        for (int b = lane; b < G * L; b += 32)
            ptab[b] = PhiloxSplit::bead_part((uint32_t)b, (uint32_t)it.chain, p.rk0, p.rk1);
        __syncwarp();
    }

    T* state = reinterpret_cast<T*>(p.state) + (ch.state_off + (int64_t)kglob * nb) * 3;
    const T* snap = reinterpret_cast<const T*>(p.snap);
    T qx[L], qy[L], qz[L];
    load_bonds<T, L>(qx, qy, qz, state, lc);

    int floored = 0;
    int s_in = (int)(p.t0 % p.S);
    int w = (int)(p.t0 / p.S);                      // window index (< 2^31)
    const uint32_t t_end = (uint32_t)(p.t0 + p.n_steps);   // steps stay below 2^32
#pragma unroll 1
    for (uint32_t t = (uint32_t)p.t0; t < t_end; ++t) {
        if (s_in == 0)   // spawn: copy the halted parent (Sec. II)
            load_bonds<T, L>(qx, qy, qz, snap + ((int64_t)(w % p.win_ring) * p.M + ch.spr_off) * 3, lc);
        floored += step_bonds<T, L, FAST, TAB>(qx, qy, qz, lc, k, (uint32_t)t, p, ptab);
        if (++s_in == p.S) {
            // one force sample per replica at the end of the evolution time
            s_in = 0;
            if (active) {
#pragma unroll
                for (int j = 0; j < L; ++j) {
                    const int i = lc.bead0 + j;
                    if (i < nb)
                        wsm[sw * nb + i] =
                            spring_tension<T, FAST>(qx[j], qy[j], qz[j], k.H, k.Hinvb, k.smin);
                }
            }
            warp_window_sum<T>(wsm, nb, it.rep_count,
                               p.part_hist + (int64_t)(w % p.win_ring) * p.part_stride + ch.part_off + (int64_t)it.group * nb);
            if (CONF && (p.flags & BD_FLAG_CONFORMATION)) {
                store_bonds<T, L>(qx, qy, qz, state, lc);
                conformation_item<T, L>(it, ch, p, w, state, sw, P, G, lc.bead0, active, kglob);
            }
            ++w;
        }
    }
    store_bonds<T, L>(qx, qy, qz, state, lc);
    if (floored) atomicAdd(p.overext + it.chain, (unsigned long long)floored);
    if (TAB) __syncwarp();     // every lane is done with ptab before the next item refills it
}

// ---------------------------------------------------------------------------
// Parents. Global warp g holds parent_warps[g].count parents (chains
// parent_items[first + s]), each on G lanes.
// Per step: update, then sample the parent's spring forces (ISF): TSF window
// sums and ISF threshold / Bell criteria. Window sums and the window's hazard
// stay in registers; the integrated hazard lives in p.lam (float64).
// ---------------------------------------------------------------------------
template <typename T, int L, bool FAST>
__global__ void __launch_bounds__(kParentThreads)
parent_kernel(const StepParams p)
{
    // per warp: the split-Philox bead parts of its parents' beads, parent s
    // at [s G L, (s + 1) G L)
    __shared__ uint4 ptab_all[kParentThreads / 32][32 * L];
    const int lane = threadIdx.x & 31;
    if ((int)(threadIdx.x >> 5) >= kParentThreads / 32) return;   // whole warps beyond the table
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (gw >= p.n_parent_warps) return;          // whole warp: no shuffle partner left behind
    const ParentWarp pw = p.parent_warps[gw];
    const int G = pw.G;
    const int P = 32 / G;
    const int sw = lane / G;
    const bool active = (sw < P) && (sw < pw.count);
    const int c = p.parent_items[pw.first + (active ? sw : 0)];
    const ChainDev ch = p.chains[c];
    const int nb = ch.N - 1;
    const LaneCtx lc = make_lane(sw < P ? lane - sw * G : 0, G, L, lane, nb, active, 0u,
                                 (uint32_t)c);
    StepConst<T, FAST> k;
    k.load(ch, p);
    uint4* ptab = ptab_all[threadIdx.x >> 5];
    for (int e = lane; e < P * G * L; e += 32) {
        const int s2 = e / (G * L);
        const int c2 = p.parent_items[pw.first + min(s2, pw.count - 1)];
        ptab[e] = PhiloxSplit::bead_part((uint32_t)(e - s2 * G * L), (uint32_t)c2, p.rk0, p.rk1);
    }
    __syncwarp();
    const uint4* my_tab = ptab + (sw < P ? sw : 0) * G * L;
    const int64_t M = p.M;
    const bool isf_thr = (p.thr_mask & BD_CRIT_ISF) != 0;
    const bool isf_bell = (p.bell_mask & BD_CRIT_ISF) != 0;
    const T fc = (T)ch.f_c;
    const double k0dt = ch.k0 * p.dt, dxs = ch.dx;

    T* state = reinterpret_cast<T*>(p.state) + ch.state_off * 3;
    T* snap = reinterpret_cast<T*>(p.snap);
    T qx[L], qy[L], qz[L];
    load_bonds<T, L>(qx, qy, qz, state, lc);

    // per-spring sampling state of this lane's springs; the Bell hazard is
    // accumulated in float64 whatever the integration precision
    T tsf[L];
    double haz[L], rem[L];
    uint32_t thr_done = 0, bell_done = 0;
#pragma unroll
    for (int j = 0; j < L; ++j) {
        const int i = lc.bead0 + j;
        const int64_t m = ch.spr_off + i;
        const bool v = active && i < nb;
        tsf[j] = v ? (T)p.tsf_acc[m] : T(0);
        haz[j] = 0.0;
        rem[j] = v ? p.exp1[CRIT_Q_ISF * M + m] - p.lam[CRIT_Q_ISF * M + m] : 0.0;
        if (!v || p.first_thr[CRIT_Q_ISF * M + m] >= 0) thr_done |= 1u << j;
        if (!v || p.first_bell[CRIT_Q_ISF * M + m] >= 0) bell_done |= 1u << j;
    }

    int floored = 0;
    int s_in = (int)(p.t0 % p.S);
    int64_t w = p.t0 / p.S;
    const int64_t t_end = p.t0 + p.n_steps;
#pragma unroll 1
    for (int64_t t = p.t0; t < t_end; ++t) {
        if (s_in == 0)   // the conformation the replicas of window w start from
            store_bonds<T, L>(qx, qy, qz, snap + ((w % p.win_ring) * M + ch.spr_off) * 3, lc);
        floored += step_bonds<T, L, FAST, true>(qx, qy, qz, lc, k, (uint32_t)t, p, my_tab);
        if (active) {
#pragma unroll
            for (int j = 0; j < L; ++j) {
                const int i = lc.bead0 + j;
                if (i < nb) {
                    const T f = spring_tension<T, FAST>(qx[j], qy[j], qz[j], k.H, k.Hinvb, k.smin);
                    tsf[j] += f;
                    if (isf_thr && !(thr_done & (1u << j)) && f >= fc) {
                        thr_done |= 1u << j;
                        p.first_thr[CRIT_Q_ISF * M + ch.spr_off + i] = t + 1;
                    }
                    if (isf_bell) {
                        haz[j] = fma(k0dt, exp(dxs * (double)f), haz[j]);
                        if (!(bell_done & (1u << j)) && haz[j] >= rem[j]) {
                            bell_done |= 1u << j;
                            p.first_bell[CRIT_Q_ISF * M + ch.spr_off + i] = t + 1;
                        }
                    }
                }
            }
        }
        if (++s_in == p.S) {
            s_in = 0;
            if (active) {
#pragma unroll
                for (int j = 0; j < L; ++j) {
                    const int i = lc.bead0 + j;
                    if (i < nb) {
                        const int64_t m = ch.spr_off + i;
                        p.tsf_hist[w * M + m] = (double)tsf[j] / (double)p.S;
                        tsf[j] = T(0);
                        if (isf_bell) {
                            const double lam = p.lam[CRIT_Q_ISF * M + m] + haz[j];
                            p.lam[CRIT_Q_ISF * M + m] = lam;
                            haz[j] = 0.0;
                            rem[j] = p.exp1[CRIT_Q_ISF * M + m] - lam;
                        }
                    }
                }
            }
            ++w;
        }
    }
    store_bonds<T, L>(qx, qy, qz, state, lc);
    if (active) {
#pragma unroll
        for (int j = 0; j < L; ++j) {
            const int i = lc.bead0 + j;
            if (i < nb) {
                const int64_t m = ch.spr_off + i;
                p.tsf_acc[m] = (double)tsf[j];
                if (isf_bell) p.lam[CRIT_Q_ISF * M + m] += haz[j];
            }
        }
    }
    if (floored) atomicAdd(p.overext + c, (unsigned long long)floored);
}

}  // namespace bdra
