// The paper's collapsed-chain model (Sec. II) in the bond layout of the
// step kernels: harmonic springs with a rest length, F = H (|Q| - r0) Q/|Q|
// (the signed force of Eq. 4 is H (|Q| - r0)), and Lennard-Jones cohesion
// between non-adjacent beads, U = u [(s/r)^12 - 2 (s/r)^6].
//
// A step of a slot (G lanes, L bonds each): the bead positions follow from
// the bonds by a prefix sum over the slot (up to a common offset, which pair
// forces do not see); the lanes of the slot exchange bead positions by
// shuffles and add the pair forces on their beads (all pairs |i - j| >= 2,
// no cutoff); the bond update of Eq. 1 then takes the difference of the
// bead forces of its two beads: Q_b += [kappa Q_b + D (Fs_{b+1} - 2 Fs_b +
// Fs_{b-1} + Flj_{b+1} - Flj_b)] dt + noise.
#pragma once

#include "bd_step.cuh"

namespace bdra {

template <typename T, bool FAST> struct Rsqrt {
    static __device__ __forceinline__ T rsqrt(T x) { return T(1) / sqrt(x); }
    static __device__ __forceinline__ T rcp(T x) { return T(1) / x; }
};
template <> struct Rsqrt<float, true> {
    static __device__ __forceinline__ float rsqrt(float x)
    {
        float r;
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
    static __device__ __forceinline__ float rcp(float x) { return rcp_approx(x); }
};

// Harmonic spring with rest length: F = c Q with c = H (1 - r0 / |Q|); a bond
// of zero length has no direction and no force.
template <typename T, bool FAST>
__device__ __forceinline__ T harmonic_coef(T qx, T qy, T qz, T H, T r0)
{
    const T q2 = bond_q2(qx, qy, qz);
    return q2 > T(0) ? H * fma(-r0, Rsqrt<T, FAST>::rsqrt(q2), T(1)) : T(0);
}

// Eq. 4: the signed spring force H (|Q| - r0).
template <typename T>
__device__ __forceinline__ T harmonic_tension(T qx, T qy, T qz, T H, T r0)
{
    return H * (sqrt(bond_q2(qx, qy, qz)) - r0);
}

// Per-chain constants of the pair forces and of the spring law with a rest
// length, in the integration precision.
template <typename T> struct LJConst {
    T r0, u12, s2;      // rest length; 12 u; s^2
    T isig, k12;        // 1 / s and 12 u / s (the pair forces in units of s)
    T fa, fb, ix2;      // vWF A2 domains: FENE and harmonic constants, 1 / x_max^2
    int N;
    bool vwf;           // BD_SPRING_VWF: even springs A2 domains, odd springs disulfide bonds
    __device__ __forceinline__ void load(const ChainDev& ch)
    {
        r0 = (T)ch.r0; u12 = (T)(12.0 * ch.lj_u); s2 = (T)ch.lj_s2; N = ch.N;
        const double sig = ch.lj_s2 > 0.0 ? sqrt(ch.lj_s2) : 1.0;
        isig = (T)(1.0 / sig); k12 = (T)(12.0 * ch.lj_u / sig);
        vwf = ch.spring == BD_SPRING_VWF;
        fa = (T)ch.vwf_fa; fb = (T)ch.vwf_fb; ix2 = (T)ch.vwf_ix2;
    }
};

// The signed force along the bond of spring i (Eq. 4) for the laws with a
// rest length: harmonic H x, x = |Q| - r0; for the vWF chain (supplementary
// material, Table S1) even springs are A2 domains, f_B x + f_A x / s with
// s = 1 - x^2 / x_max^2 floored at smin (counted in floored), odd springs
// disulfide bonds H x.
template <typename T, bool FAST>
__device__ __forceinline__ T rest_law_force(T q, bool a2, T H, const LJConst<T>& kl, T smin, int& floored)
{
    const T x = q - kl.r0;
    if (!kl.vwf || !a2) return H * x;
    const T s = fma(-x * x, kl.ix2, T(1));
    floored += s < smin;
    return fma(kl.fb, x, Div<T, FAST>::div(kl.fa * x, fmax(s, smin)));
}

// The same as a coefficient c of F = c Q (zero for a bond of zero length).
template <typename T, bool FAST>
__device__ __forceinline__ T rest_law_coef(T qx, T qy, T qz, bool a2, T H, const LJConst<T>& kl, T smin,
                                           int& floored)
{
    if (!kl.vwf) return harmonic_coef<T, FAST>(qx, qy, qz, H, kl.r0);
    const T q2 = bond_q2(qx, qy, qz);
    if (!(q2 > T(0))) return T(0);
    const T iq = Rsqrt<T, FAST>::rsqrt(q2);
    return rest_law_force<T, FAST>(q2 * iq, a2, H, kl, smin, floored) * iq;
}

template <typename T, bool FAST>
__device__ __forceinline__ T rest_law_tension(T qx, T qy, T qz, bool a2, T H, const LJConst<T>& kl, T smin)
{
    int dummy = 0;
    return rest_law_force<T, FAST>(sqrt(bond_q2(qx, qy, qz)), a2, H, kl, smin, dummy);
}

// Inclusive prefix sum over the lanes of a slot (seg: the lane's position in
// its slot; lanes outside slots pass seg 0 and get junk they never use).
template <typename T>
__device__ __forceinline__ T lj_slot_scan(T v, int seg)
{
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const T u = __shfl_up_sync(0xffffffffu, v, d);
        if (seg >= d) v += u;
    }
    return v;
}

// Beads that take no part in pair forces (the padding beads of a ragged
// slot, the partners of a lane that skips a block) are moved this far away:
// their Lennard-Jones terms underflow (float: to zero; double: below one
// rounding unit of any force), so no pair needs a mask.
template <typename T> __device__ __forceinline__ T lj_far() { return T(1e12); }

// The pair force between bead a (mine) and bead b: c = 12 u (x^6 - x^12) / r^2
// with x = s / r, so that c d (d = r_b - r_a) is the force on a and -c d the
// force on b.
template <typename T, bool FAST>
__device__ __forceinline__ T lj_coef(T dx, T dy, T dz, const LJConst<T>& kl)
{
    const T ir2 = Rsqrt<T, FAST>::rcp(fma(dx, dx, fma(dy, dy, dz * dz)));
    const T x2 = kl.s2 * ir2;
    const T x6 = x2 * x2 * x2;
    return fma(-x6, x6, x6) * (kl.u12 * ir2);
}

// The same force for a separation d' = d / s in units of s: with x = 1/|d'|,
// c' = x^8 - x^14 and the force on a is (12 u / s) c' d' (kl.k12, applied
// once per bead after the pair sums). One multiply a pair fewer than the
// unscaled form.
template <typename T, bool FAST>
__device__ __forceinline__ T lj_coef_scaled(T dx, T dy, T dz)
{
    const T ir2 = Rsqrt<T, FAST>::rcp(fma(dx, dx, fma(dy, dy, dz * dz)));
    const T x4 = ir2 * ir2;
    const T x6 = x4 * ir2;
    const T x8 = x4 * x4;
    return fma(-x8, x6, x8);
}

// The ring part of the pair forces (d = 1 .. G/2, as in step_bonds_lj) with
// the float32 arithmetic of two of the lane's beads at a time in packed
// two-wide instructions (FFMA2 / FMUL2): the lane's beads 2jp and 2jp+1
// against one partner bead; an odd last bead goes alone. Each half rounds
// as the scalar form; only the order of the partner reaction's sum differs.
template <int L>
__device__ __forceinline__ void lj_ring_pairs_packed(const float (&px)[L], const float (&py)[L], const float (&pz)[L],
                                                     float (&gx)[L], float (&gy)[L], float (&gz)[L],
                                                     const LJConst<float>& kl, bool in_slot, int seg, int G,
                                                     int slot_base)
{
    constexpr int LP = L / 2;
    const int lane = threadIdx.x & 31;
    const float2 m1 = make_float2(-1.0f, -1.0f);

    float2 gx2[LP], gy2[LP], gz2[LP];
#pragma unroll
    for (int jp = 0; jp < LP; ++jp) gx2[jp] = gy2[jp] = gz2[jp] = make_float2(0.0f, 0.0f);
    const int half = G >> 1;
#pragma unroll 1
    for (int d = 1; d <= half; ++d) {
        int pf = seg + d;
        if (pf >= G) pf -= G;
        int pb = seg - d;
        if (pb < 0) pb += G;
        const int srcf = in_slot ? slot_base + pf : lane;    // < 32: slots fit the warp
        const int srcb = in_slot ? slot_base + pb : lane;
        const bool skip = 2 * d == G && seg >= half;
        const bool bonded = d == 1 && seg + 1 < G;          // my last bead - its first bead
#pragma unroll
        for (int kk = 0; kk < L; ++kk) {
            float bx = __shfl_sync(0xffffffffu, px[kk], srcf);
            const float by = __shfl_sync(0xffffffffu, py[kk], srcf);
            const float bz = __shfl_sync(0xffffffffu, pz[kk], srcf);
            if (skip) bx = -lj_far<float>() * 1000.0f;
            const float2 Bx = make_float2(bx, bx), By = make_float2(by, by), Bz = make_float2(bz, bz);
            float2 hx2 = make_float2(0.0f, 0.0f), hy2 = hx2, hz2 = hx2;
#pragma unroll
            for (int jp = 0; jp < LP; ++jp) {
                const float2 dx = __ffma2_rn(make_float2(px[2 * jp], px[2 * jp + 1]), m1, Bx);
                const float2 dy = __ffma2_rn(make_float2(py[2 * jp], py[2 * jp + 1]), m1, By);
                const float2 dz = __ffma2_rn(make_float2(pz[2 * jp], pz[2 * jp + 1]), m1, Bz);
                const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
                const float2 ir2 = make_float2(rcp_approx(r2.x), rcp_approx(r2.y));
                const float2 x4 = __fmul2_rn(ir2, ir2);
                const float2 x6 = __fmul2_rn(x4, ir2);
                const float2 x8 = __fmul2_rn(x4, x4);
                float2 c = __ffma2_rn(make_float2(-x8.x, -x8.y), x6, x8);
                if (kk == 0 && 2 * jp + 1 == L - 1 && bonded) c.y = 0.0f;
                gx2[jp] = __ffma2_rn(c, dx, gx2[jp]);
                gy2[jp] = __ffma2_rn(c, dy, gy2[jp]);
                gz2[jp] = __ffma2_rn(c, dz, gz2[jp]);
                hx2 = __ffma2_rn(c, dx, hx2);
                hy2 = __ffma2_rn(c, dy, hy2);
                hz2 = __ffma2_rn(c, dz, hz2);
            }
            float hx = hx2.x + hx2.y, hy = hy2.x + hy2.y, hz = hz2.x + hz2.y;
            if constexpr (L & 1) {
                const float dx = bx - px[L - 1], dy = by - py[L - 1], dz = bz - pz[L - 1];
                float c = lj_coef_scaled<float, true>(dx, dy, dz);
                if (kk == 0 && bonded) c = 0.0f;
                gx[L - 1] = fmaf(c, dx, gx[L - 1]); gy[L - 1] = fmaf(c, dy, gy[L - 1]); gz[L - 1] = fmaf(c, dz, gz[L - 1]);
                hx = fmaf(c, dx, hx); hy = fmaf(c, dy, hy); hz = fmaf(c, dz, hz);
            }
            // the reaction on bead kk of this lane, from the lane d places back
            gx[kk] -= __shfl_sync(0xffffffffu, hx, srcb);
            gy[kk] -= __shfl_sync(0xffffffffu, hy, srcb);
            gz[kk] -= __shfl_sync(0xffffffffu, hz, srcb);
        }
    }
#pragma unroll
    for (int jp = 0; jp < LP; ++jp) {
        gx[2 * jp] += gx2[jp].x; gx[2 * jp + 1] += gx2[jp].y;
        gy[2 * jp] += gy2[jp].x; gy[2 * jp + 1] += gy2[jp].y;
        gz[2 * jp] += gz2[jp].x; gz[2 * jp + 1] += gz2[jp].y;
    }
}

// One Eq. 1 step of the lane's L bonds of a collapsed chain. in_slot: the
// lane belongs to a slot, slot_base its first lane, seg its position in it, G
// the lanes per slot. Every lane of the warp calls it.
//
// Pair forces: every non-adjacent pair once (Newton's third law). A lane's
// own beads pair among themselves (k >= j + 2); for d = 1 .. G/2 a lane
// pairs its beads with those of the lane d places further round the slot's
// ring, keeps the forces on its beads and shuffles the reactions back to
// that lane. Every lane pair of the ring is at one cyclic distance d <= G/2
// from exactly one of its two lanes, except at d = G/2 for even G, which
// only the first half of the ring takes. Beads of different lanes are
// adjacent only across the boundary to the next lane (d = 1, no wrap).
// H: the slot's noise half at compile time (-1: lc.noise_half).
template <typename T, int L, bool FAST, bool TAB, int H = -1>
__device__ __forceinline__ int step_bonds_lj(T (&qx)[L], T (&qy)[L], T (&qz)[L], const LaneCtx& lc,
                                             const StepConst<T, FAST>& k, const LJConst<T>& kl,
                                             bool in_slot, int seg, int G, int slot_base,
                                             uint32_t step, const StepParams& p, const uint4* ptab)
{
    const int lane = threadIdx.x & 31;
    int floored = 0;
    // spring forces of the lane's bonds (bond b joins beads b and b+1)
    T fx[L], fy[L], fz[L];
#pragma unroll
    for (int j = 0; j < L; ++j) {
        int fl = 0;
        const T c = rest_law_coef<T, FAST>(qx[j], qy[j], qz[j], ((lc.bead0 + j) & 1) == 0, k.H, kl, k.smin, fl);
        if (j < lc.nv) floored += fl;
        fx[j] = c * qx[j]; fy[j] = c * qy[j]; fz[j] = c * qz[j];
    }
    // bead positions (common offset dropped): exclusive prefix over the slot
    T px[L], py[L], pz[L];
    {
        T sx = T(0), sy = T(0), sz = T(0);
#pragma unroll
        for (int j = 0; j < L; ++j) { sx += qx[j]; sy += qy[j]; sz += qz[j]; }
        T x = lj_slot_scan(sx, seg) - sx, y = lj_slot_scan(sy, seg) - sy, z = lj_slot_scan(sz, seg) - sz;
#pragma unroll
        for (int j = 0; j < L; ++j) {
            const bool real = lc.bead0 + j < kl.N;
            px[j] = real ? x * kl.isig : lj_far<T>() * (T)(lc.bead0 + j + 1);   // in units of s
            py[j] = real ? y * kl.isig : T(0);
            pz[j] = real ? z * kl.isig : T(0);
            x += qx[j]; y += qy[j]; z += qz[j];
        }
    }
    T gx[L], gy[L], gz[L];
#pragma unroll
    for (int j = 0; j < L; ++j) gx[j] = gy[j] = gz[j] = T(0);
    // the lane's own pairs
#pragma unroll
    for (int j = 0; j < L; ++j)
#pragma unroll
        for (int kk = j + 2; kk < L; ++kk) {
            const T dx = px[kk] - px[j], dy = py[kk] - py[j], dz = pz[kk] - pz[j];
            const T c = lj_coef_scaled<T, FAST>(dx, dy, dz);
            gx[j] = fma(c, dx, gx[j]); gy[j] = fma(c, dy, gy[j]); gz[j] = fma(c, dz, gz[j]);
            gx[kk] = fma(-c, dx, gx[kk]); gy[kk] = fma(-c, dy, gy[kk]); gz[kk] = fma(-c, dz, gz[kk]);
        }
    // pairs with the lanes d places round the ring
    const int half = G >> 1;
    if constexpr (sizeof(T) == 4 && FAST && L >= 2) {
        lj_ring_pairs_packed<L>(px, py, pz, gx, gy, gz, kl, in_slot, seg, G, slot_base);
    } else {
#pragma unroll 1
    for (int d = 1; d <= half; ++d) {
        int pf = seg + d;
        if (pf >= G) pf -= G;
        int pb = seg - d;
        if (pb < 0) pb += G;
        const int srcf = in_slot ? slot_base + pf : lane;    // < 32: slots fit the warp
        const int srcb = in_slot ? slot_base + pb : lane;
        const bool skip = 2 * d == G && seg >= half;
        const bool bonded = d == 1 && seg + 1 < G;          // my last bead - its first bead
#pragma unroll
        for (int kk = 0; kk < L; ++kk) {
            T bx = __shfl_sync(0xffffffffu, px[kk], srcf);
            const T by = __shfl_sync(0xffffffffu, py[kk], srcf);
            const T bz = __shfl_sync(0xffffffffu, pz[kk], srcf);
            if (skip) bx = -lj_far<T>() * T(1000);
            T hx = T(0), hy = T(0), hz = T(0);
#pragma unroll
            for (int j = 0; j < L; ++j) {
                const T dx = bx - px[j], dy = by - py[j], dz = bz - pz[j];
                T c = lj_coef_scaled<T, FAST>(dx, dy, dz);
                if (kk == 0 && j == L - 1 && bonded) c = T(0);
                gx[j] = fma(c, dx, gx[j]); gy[j] = fma(c, dy, gy[j]); gz[j] = fma(c, dz, gz[j]);
                hx = fma(c, dx, hx); hy = fma(c, dy, hy); hz = fma(c, dz, hz);
            }
            // the reaction on bead kk of this lane, from the lane d places back
            gx[kk] -= __shfl_sync(0xffffffffu, hx, srcb);
            gy[kk] -= __shfl_sync(0xffffffffu, hy, srcb);
            gz[kk] -= __shfl_sync(0xffffffffu, hz, srcb);
        }
    }
    }
#pragma unroll
    for (int j = 0; j < L; ++j) { gx[j] *= kl.k12; gy[j] *= kl.k12; gz[j] *= kl.k12; }
    // halo: spring force of the previous lane's last bond and the next lane's
    // first bond; the next lane's first-bead pair force and noise
    T fmx = shfl(fx[L - 1], lc.src_prev), fmy = shfl(fy[L - 1], lc.src_prev), fmz = shfl(fz[L - 1], lc.src_prev);
    T fnx = shfl(fx[0], lc.src_next), fny = shfl(fy[0], lc.src_next), fnz = shfl(fz[0], lc.src_next);
    T gnx = shfl(gx[0], lc.src_next), gny = shfl(gy[0], lc.src_next), gnz = shfl(gz[0], lc.src_next);
    if (!lc.has_prev) { fmx = T(0); fmy = T(0); fmz = T(0); }
    if (!lc.has_next) { fnx = T(0); fny = T(0); fnz = T(0); gnx = T(0); gny = T(0); gnz = T(0); }
    uint3 sp = make_uint3(0u, 0u, 0u);
    if (TAB) sp = PhiloxSplit::step_part(step, lc.noise_word, p.rk0);
    T xcx, xcy, xcz;
    if (TAB) bead_noise_split<T, FAST, H>(ptab[lc.bead0], sp, p, lc.noise_half, xcx, xcy, xcz);
    else bead_noise<T, FAST, H>((uint32_t)lc.bead0, lc.slot_key, step, lc.chain, p, xcx, xcy, xcz);
    const T hx = shfl(xcx, lc.src_next), hy = shfl(xcy, lc.src_next), hz = shfl(xcz, lc.src_next);
#pragma unroll
    for (int j = 0; j < L; ++j) {
        T xnx, xny, xnz, fpx, fpy, fpz, ghx, ghy, ghz;
        if (j + 1 < L) {
            uint32_t bj = (uint32_t)(lc.bead0 + j + 1);
            asm volatile("" : "+r"(bj));     // keep per-bead noise work inside the step loop
            if (TAB) bead_noise_split<T, FAST, H>(ptab[bj], sp, p, lc.noise_half, xnx, xny, xnz);
            else bead_noise<T, FAST, H>(bj, lc.slot_key, step, lc.chain, p, xnx, xny, xnz);
            fpx = fx[j + 1]; fpy = fy[j + 1]; fpz = fz[j + 1];
            ghx = gx[j + 1]; ghy = gy[j + 1]; ghz = gz[j + 1];
        } else {
            xnx = hx; xny = hy; xnz = hz;
            fpx = fnx; fpy = fny; fpz = fnz;
            ghx = gnx; ghy = gny; ghz = gnz;
        }
        if (j < lc.nv) {
            const T lx = fma(T(-2), fx[j], fpx + fmx) + (ghx - gx[j]);
            const T ly = fma(T(-2), fy[j], fpy + fmy) + (ghy - gy[j]);
            const T lz = fma(T(-2), fz[j], fpz + fmz) + (ghz - gz[j]);
            const T ox = qx[j], oy = qy[j], oz = qz[j];
            qx[j] = fma(k.cn, xnx - xcx, fma(k.cd, lx, fma(k.axz, oz, fma(k.axx, ox, ox))));
            qy[j] = fma(k.cn, xny - xcy, fma(k.cd, ly, fma(k.ayy, oy, oy)));
            qz[j] = fma(k.cn, xnz - xcz, fma(k.cd, lz, fma(k.azz, oz, oz)));
        }
        fmx = fx[j]; fmy = fy[j]; fmz = fz[j];
        xcx = xnx; xcy = xny; xcz = xnz;
    }
    return floored;
}

}  // namespace bdra
