// Replica kernel with two replicas per lane (float32 only).
//
// Same method and the same rounding sequence as replica_kernel<float, L,
// true> (bd_window.cuh), but every lane carries replicas 2s+1 and 2s+2 of the
// same L springs side by side in float2 registers, so the float32 arithmetic
// of a step (spring law, Laplacian, update, Box-Muller products) issues as
// packed two-wide instructions (FFMA2 / FADD2 / FMUL2 on sm_100-class SMs).
// When the two replicas are a noise pair (2j - 1, 2j), one Philox call per
// bead and step gives both their normals; the special-function work stays
// per normal. A packed
// operation rounds each half exactly like its scalar form, and a - b is
// written fma(b, -1, a) (exact product, one rounding), so both layouts give
// bitwise-equal results.
#pragma once

#include "bd_window.cuh"

namespace bdra {

// Which groups of the step's float32 operations issue as packed two-wide
// instructions (the others issue as two scalar ones; both forms round
// identically, so the choice never changes a result). A packed operation
// occupies both halves of the FMA pipe, and the heavy half is also where the
// Philox 32 x 32 -> 64 multiplies run, so packing saves issue slots at the
// price of heavy-pipe cycles; the mask sets the balance.
#ifndef BD_PACK_MASK
#define BD_PACK_MASK 31
#endif
enum { PK_UNIF = 1, PK_BM = 2, PK_SPRING = 4, PK_LAP = 8, PK_UPD = 16 };
// 1: the per-bead noise work stays where it is written in the step loop (an
// empty asm fence on the bead index); 0: the compiler may move it (measured
// 1% faster with one generator call per replica pair; same results).
#ifndef BD_PAIR_NOISE_FENCE
#define BD_PAIR_NOISE_FENCE 0
#endif

template <int GROUP>
struct F2G {
    static constexpr bool packed = (BD_PACK_MASK & GROUP) != 0;
    static __device__ __forceinline__ float2 add(float2 a, float2 b)
    {
        if (packed) return __fadd2_rn(a, b);
        return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y));
    }
    static __device__ __forceinline__ float2 mul(float2 a, float2 b)
    {
        if (packed) return __fmul2_rn(a, b);
        return make_float2(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y));
    }
    static __device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c)
    {
        if (packed) return __ffma2_rn(a, b, c);
        return make_float2(__fmaf_rn(a.x, b.x, c.x), __fmaf_rn(a.y, b.y, c.y));
    }
    // a - b as fma(b, -1, a): exact product, one rounding
    static __device__ __forceinline__ float2 sub(float2 a, float2 b)
    {
        return fma(b, make_float2(-1.0f, -1.0f), a);
    }
};

struct F2 {
    static __device__ __forceinline__ float2 splat(float a) { return make_float2(a, a); }
};
using F2U = F2G<PK_UNIF>;
using F2B = F2G<PK_BM>;
using F2S = F2G<PK_SPRING>;
using F2L = F2G<PK_LAP>;
using F2P = F2G<PK_UPD>;

// Spring coefficient H / s for both halves; floor counts per half.
__device__ __forceinline__ float2 spring_coef2(float2 qx, float2 qy, float2 qz, float2 H2,
                                               float2 nHinvb2, float smin, int& fla, int& flb)
{
    const float2 q2 = F2S::fma(qx, qx, F2S::fma(qy, qy, F2S::mul(qz, qz)));
    const float2 s = F2S::fma(nHinvb2, q2, F2::splat(1.0f));
    fla += s.x < smin;
    flb += s.y < smin;
    return F2S::mul(H2, make_float2(rcp_approx(fmaxf(s.x, smin)), rcp_approx(fmaxf(s.y, smin))));
}

// Box-Muller of one Philox output for a replica pair: .x the first half
// (z0, z1, z2) and .y the second (z3, z4, z5) of Normals<float, true>::draw,
// bitwise (the packed operations round each half like the scalar ones, and
// a - b is fma(b, -1, a), one rounding like __fsub_rn). Sign-flipped normals
// (see Normals<float, true>::sign).
__device__ __forceinline__ void box_muller_pair(uint4 x, float2& z0, float2& z1, float2& z2)
{
    const float2 u02 = F2U::sub(make_float2(Fields21::one_plus(x, 0), Fields21::one_plus(x, 2)),
                                F2::splat(FastBM::rad_off));
    const float u4 = __fsub_rn(Fields21::one_plus(x, 4), FastBM::rad_off);
    const float2 a02 = F2B::mul(F2::splat(FastBM::m2ln2), make_float2(lg2_approx(u02.x), lg2_approx(u02.y)));
    const float a4 = __fmul_rn(FastBM::m2ln2, lg2_approx(u4));
    const float r0 = sqrt_approx(fabsf(a02.x)), r2 = sqrt_approx(fabsf(a02.y)), r4 = sqrt_approx(fabsf(a4));
    const float2 t13 = F2U::fma(make_float2(Fields21::one_plus(x, 1), Fields21::one_plus(x, 3)),
                                F2::splat(FastBM::twopi), F2::splat(FastBM::off));
    const float t5 = __fmaf_rn(Fields21::one_plus(x, 5), FastBM::twopi, FastBM::off);
    z0 = F2B::mul(make_float2(r0, r2), make_float2(cos_approx(t13.x), sin_approx(t13.y)));
    z1 = F2B::mul(make_float2(r0, r4), make_float2(sin_approx(t13.x), cos_approx(t5)));
    z2 = F2B::mul(make_float2(r2, r4), make_float2(cos_approx(t13.y), sin_approx(t5)));
}

// Noise of one bead for both replicas of the lane. SHARED: the lane's two
// slots form one replica pair (noise word wa, halves 0 and 1), one generator
// call. Otherwise each slot draws its own call and half (identical-noise
// runs, or a pair split across work items). With a bead table (TAB) the
// Philox rounds that depend only on (bead, chain) come from ptab[bead] and
// those that depend only on (step, noise word) from spa / spb
// (PhiloxSplit); otherwise the full generator runs.
template <bool TAB, bool SHARED>
__device__ __forceinline__ void bead_noise2(uint32_t bead, uint32_t wa, uint32_t ha, uint32_t wb,
                                            uint32_t hb, uint32_t step, uint32_t chain,
                                            const StepParams& p, const uint4* ptab, uint3 spa,
                                            uint3 spb, float2& z0, float2& z1, float2& z2)
{
    if (SHARED) {
        const uint4 x = TAB ? PhiloxSplit::finish(ptab[bead], spa, p.rk0, p.rk1)
                            : philox4x32_10_rk(make_uint4(bead, wa, step, chain), p.rk0, p.rk1);
        box_muller_pair(x, z0, z1, z2);
    } else {
        uint4 xa, xb;
        if (TAB) {
            const uint4 bp = ptab[bead];
            xa = PhiloxSplit::finish(bp, spa, p.rk0, p.rk1);
            xb = PhiloxSplit::finish(bp, spb, p.rk0, p.rk1);
        } else {
            xa = philox4x32_10_rk(make_uint4(bead, wa, step, chain), p.rk0, p.rk1);
            xb = philox4x32_10_rk(make_uint4(bead, wb, step, chain), p.rk0, p.rk1);
        }
        Normals<float, true>::draw(xa, ha, z0.x, z1.x, z2.x);
        Normals<float, true>::draw(xb, hb, z0.y, z1.y, z2.y);
    }
}

__device__ __forceinline__ float2 shfl2(float2 v, int src)
{
    return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// Packed per-chain constants.
struct StepConst2 {
    float2 H, nHinvb, cd, cn, axx, ayy, azz, axz;
    float smin;
    __device__ __forceinline__ void load(const ChainDev& ch, const StepParams& p)
    {
        StepConst<float, true> k;
        k.load(ch, p);
        H = F2::splat(k.H); nHinvb = F2::splat(-k.Hinvb); cd = F2::splat(k.cd); cn = F2::splat(k.cn);
        axx = F2::splat(k.axx); ayy = F2::splat(k.ayy); azz = F2::splat(k.azz); axz = F2::splat(k.axz);
        smin = k.smin;
    }
};

// One Eq. 1 step (bond form) of both replicas' L bonds; all lanes call it.
// Replica a is the lane's slot (lc), replica b the slot kb.
template <int L, bool TAB, bool SHARED>
__device__ __forceinline__ void step_bonds2(float2 (&qx)[L], float2 (&qy)[L], float2 (&qz)[L],
                                            const LaneCtx& lc, uint32_t kb, bool act_b,
                                            const StepConst2& k, uint32_t step,
                                            const StepParams& p, const uint4* ptab, int& fl_out)
{
    const uint32_t wb = noise_word(kb), hb = noise_half(kb);
    uint3 spa = make_uint3(0u, 0u, 0u), spb = spa;
    if (TAB) {
        spa = PhiloxSplit::step_part(step, lc.noise_word, p.rk0);
        if (!SHARED) spb = PhiloxSplit::step_part(step, wb, p.rk0);
    }
    int fla = 0, flb = 0;
    const float2 c0 = spring_coef2(qx[0], qy[0], qz[0], k.H, k.nHinvb, k.smin, fla, flb);
    const float2 f0x = F2S::mul(c0, qx[0]), f0y = F2S::mul(c0, qy[0]), f0z = F2S::mul(c0, qz[0]);
    float2 fLx = f0x, fLy = f0y, fLz = f0z;
    if (L > 1) {
        const float2 cL = spring_coef2(qx[L - 1], qy[L - 1], qz[L - 1], k.H, k.nHinvb, k.smin, fla, flb);
        fLx = F2S::mul(cL, qx[L - 1]); fLy = F2S::mul(cL, qy[L - 1]); fLz = F2S::mul(cL, qz[L - 1]);
    }
    float2 fmx = shfl2(fLx, lc.src_prev), fmy = shfl2(fLy, lc.src_prev), fmz = shfl2(fLz, lc.src_prev);
    float2 fnx = shfl2(f0x, lc.src_next), fny = shfl2(f0y, lc.src_next), fnz = shfl2(f0z, lc.src_next);
    const float2 zero = F2::splat(0.0f);
    if (!lc.has_prev) { fmx = zero; fmy = zero; fmz = zero; }
    if (!lc.has_next) { fnx = zero; fny = zero; fnz = zero; }
    float2 xcx, xcy, xcz;
    bead_noise2<TAB, SHARED>((uint32_t)lc.bead0, lc.noise_word, lc.noise_half, wb, hb, step, lc.chain, p,
                             ptab, spa, spb, xcx, xcy, xcz);
    const float2 hx = shfl2(xcx, lc.src_next), hy = shfl2(xcy, lc.src_next), hz = shfl2(xcz, lc.src_next);
    const float2 m2 = F2::splat(-2.0f);

    float2 fcx = f0x, fcy = f0y, fcz = f0z;
#pragma unroll
    for (int j = 0; j < L; ++j) {
        float2 fpx, fpy, fpz, xnx, xny, xnz;
        if (j + 1 < L) {
            if (j + 1 == L - 1) {
                fpx = fLx; fpy = fLy; fpz = fLz;
            } else {
                const float2 c = spring_coef2(qx[j + 1], qy[j + 1], qz[j + 1], k.H, k.nHinvb, k.smin, fla, flb);
                fpx = F2S::mul(c, qx[j + 1]); fpy = F2S::mul(c, qy[j + 1]); fpz = F2S::mul(c, qz[j + 1]);
            }
            uint32_t bj = (uint32_t)(lc.bead0 + j + 1);
#if BD_PAIR_NOISE_FENCE
            asm volatile("" : "+r"(bj));     // keep per-bead Philox work inside the step loop
#endif
            bead_noise2<TAB, SHARED>(bj, lc.noise_word, lc.noise_half, wb, hb, step, lc.chain, p, ptab,
                                     spa, spb, xnx, xny, xnz);
        } else {
            fpx = fnx; fpy = fny; fpz = fnz;
            xnx = hx; xny = hy; xnz = hz;
        }
        if (j < lc.nv) {
            const float2 lx = F2L::fma(m2, fcx, F2L::add(fpx, fmx));
            const float2 ly = F2L::fma(m2, fcy, F2L::add(fpy, fmy));
            const float2 lz = F2L::fma(m2, fcz, F2L::add(fpz, fmz));
            const float2 ox = qx[j], oy = qy[j], oz = qz[j];
            qx[j] = F2P::fma(k.cn, F2P::sub(xnx, xcx), F2P::fma(k.cd, lx, F2P::fma(k.axz, oz, F2P::fma(k.axx, ox, ox))));
            qy[j] = F2P::fma(k.cn, F2P::sub(xny, xcy), F2P::fma(k.cd, ly, F2P::fma(k.ayy, oy, oy)));
            qz[j] = F2P::fma(k.cn, F2P::sub(xnz, xcz), F2P::fma(k.cd, lz, F2P::fma(k.azz, oz, oz)));
        }
        fmx = fcx; fmy = fcy; fmz = fcz;
        fcx = fpx; fcy = fpy; fcz = fpz;
        xcx = xnx; xcy = xny; xcz = xnz;
    }
    fl_out += lc.active ? fla + (act_b ? flb : 0) : 0;
}

// Eq. 5 diagnostics of a work item with two replicas per lane at the end of
// window w; their bonds were just stored at sa / sb.
template <int L>
__device__ __noinline__ void conformation_pair(const ItemDev& it, const ChainDev& ch,
                                               const StepParams& p, int w, const float* sa,
                                               const float* sb, int sw, int P, int G, int bead0,
                                               bool act_a, bool act_b, int ka, int kb)
{
    const SlotRun r = slot_run((int)(threadIdx.x & 31), sw, P, G);
    const float* pc = reinterpret_cast<const float*>(p.snap) + ((int64_t)(w % p.win_ring) * p.M + ch.spr_off) * 3;
    float acc[L][3];
#pragma unroll
    for (int j = 0; j < L; ++j) acc[j][0] = acc[j][1] = acc[j][2] = float(0);
    eq5_replica<float, L>(sa, pc, bead0, r, ch.N, act_a, acc,
                          p.dbar + ((int64_t)w * p.n_rep + ch.rep_off + ka - 1) * 3);
    eq5_replica<float, L>(sb, pc, bead0, r, ch.N, act_b, acc,
                          p.dbar + ((int64_t)w * p.n_rep + ch.rep_off + kb - 1) * 3);
    if (it.group == 0)
        eq5_rgz<float, L>(pc, bead0, r, ch.N, sw == 0, p.rgz + (int64_t)w * p.n_chains + it.chain);
    eq5_beads_out<float, L>(acc, bead0, r, sw, P, ch.N, (it.rep_count + 1) / 2,
                     p.dbead_part + ((int64_t)(w % p.win_ring) * p.bpart_stride + ch.bpart_off +
                                     (int64_t)it.group * ch.N) * 3);
}

// One warp work item with two replicas per lane: lane run s holds replicas
// rep_begin + 2s + 1 (.x) and rep_begin + 2s + 2 (.y). With TAB, ptab is
// this warp's table of 32 L bead parts of the Philox counter. CONF compiles
// in the Eq. 5 window-end diagnostics. SHARED: the lane's two replicas are a
// noise pair (one generator call per bead and step).
template <int L, bool TAB, bool CONF, bool SHARED>
__device__ __forceinline__ void run_pair_item_k(const ItemDev& it, const StepParams& p, float* wsm,
                                                uint4* ptab)
{
    const ChainDev ch = p.chains[it.chain];
    const int nb = ch.N - 1;
    const int G = (ch.N + L - 1) / L;
    const int P = 32 / G;
    const int lane = threadIdx.x & 31;
    const int sw = lane / G;
    const int ra = 2 * sw, rb = 2 * sw + 1;                 // replica slots of this item
    const bool act_a = (sw < P) && (ra < it.rep_count);
    const bool act_b = (sw < P) && (rb < it.rep_count);
    const int ka = it.rep_begin + ra + 1, kb = it.rep_begin + rb + 1;
    const bool same = (p.flags & BD_FLAG_IDENTICAL_NOISE) != 0;
    const LaneCtx lc = make_lane(sw < P ? lane - sw * G : 0, G, L, lane, nb, act_a,
                                 same ? 0u : (uint32_t)ka, (uint32_t)it.chain + p.chain_base);
    const uint32_t keyb = same ? 0u : (uint32_t)kb;
    StepConst2 k;
    k.load(ch, p);
    if (TAB) {       // bead parts of the noise counter for every bead a lane of this chain draws
        for (int b = lane; b < G * L; b += 32)
            ptab[b] = PhiloxSplit::bead_part((uint32_t)b, (uint32_t)it.chain + p.chain_base, p.rk0, p.rk1);
        __syncwarp();
    }

    float* state = reinterpret_cast<float*>(p.state) + ch.state_off * 3;
    float* sa = state + (int64_t)ka * nb * 3;
    float* sb = state + (int64_t)kb * nb * 3;
    const float* snap = reinterpret_cast<const float*>(p.snap);
    float2 qx[L], qy[L], qz[L];
#pragma unroll
    for (int j = 0; j < L; ++j) {
        const int i = lc.bead0 + j;
        const bool v = i < nb;
        qx[j] = make_float2(v && act_a ? sa[3 * i] : 0.0f, v && act_b ? sb[3 * i] : 0.0f);
        qy[j] = make_float2(v && act_a ? sa[3 * i + 1] : 0.0f, v && act_b ? sb[3 * i + 1] : 0.0f);
        qz[j] = make_float2(v && act_a ? sa[3 * i + 2] : 0.0f, v && act_b ? sb[3 * i + 2] : 0.0f);
    }

    int floored = 0;
    int s_in = (int)(p.t0 % p.S);
    int w = (int)(p.t0 / p.S);                      // window index (< 2^31)
    const uint32_t t_end = (uint32_t)(p.t0 + p.n_steps);   // steps stay below 2^32
#pragma unroll 1
    for (uint32_t t = (uint32_t)p.t0; t < t_end; ++t) {
        if (s_in == 0) {  // spawn both replicas from the halted parent (Sec. II)
            const float* src = snap + ((int64_t)(w % p.win_ring) * p.M + ch.spr_off) * 3;
#pragma unroll
            for (int j = 0; j < L; ++j) {
                const int i = lc.bead0 + j;
                if (act_a && i < nb) {
                    const float x = src[3 * i], y = src[3 * i + 1], z = src[3 * i + 2];
                    qx[j] = make_float2(x, x); qy[j] = make_float2(y, y); qz[j] = make_float2(z, z);
                }
            }
        }
        step_bonds2<L, TAB, SHARED>(qx, qy, qz, lc, keyb, act_b, k, (uint32_t)t, p, ptab, floored);
        if (++s_in == p.S) {
            s_in = 0;
            if (act_a) {
#pragma unroll
                for (int j = 0; j < L; ++j) {
                    const int i = lc.bead0 + j;
                    if (i < nb) {
                        wsm[ra * nb + i] = spring_tension<float, true>(qx[j].x, qy[j].x, qz[j].x, k.H.x, -k.nHinvb.x, k.smin);
                        if (act_b)
                            wsm[rb * nb + i] = spring_tension<float, true>(qx[j].y, qy[j].y, qz[j].y, k.H.y, -k.nHinvb.y, k.smin);
                    }
                }
            }
            warp_window_sum<float>(wsm, nb, it.rep_count,
                                   p.part_hist + (int64_t)(w % p.win_ring) * p.part_stride + ch.part_off + (int64_t)it.group * nb);
            if (CONF && (p.flags & BD_FLAG_CONFORMATION)) {
#pragma unroll
                for (int j = 0; j < L; ++j) {
                    const int i = lc.bead0 + j;
                    if (i < nb) {
                        if (act_a) { sa[3 * i] = qx[j].x; sa[3 * i + 1] = qy[j].x; sa[3 * i + 2] = qz[j].x; }
                        if (act_b) { sb[3 * i] = qx[j].y; sb[3 * i + 1] = qy[j].y; sb[3 * i + 2] = qz[j].y; }
                    }
                }
                conformation_pair<L>(it, ch, p, w, sa, sb, sw, P, G, lc.bead0, act_a, act_b, ka, kb);
            }
            ++w;
        }
    }
#pragma unroll
    for (int j = 0; j < L; ++j) {
        const int i = lc.bead0 + j;
        if (i < nb) {
            if (act_a) { sa[3 * i] = qx[j].x; sa[3 * i + 1] = qy[j].x; sa[3 * i + 2] = qz[j].x; }
            if (act_b) { sb[3 * i] = qx[j].y; sb[3 * i + 1] = qy[j].y; sb[3 * i + 2] = qz[j].y; }
        }
    }
    if (floored) atomicAdd(p.overext + it.chain, (unsigned long long)floored);
    if (TAB) __syncwarp();     // every lane is done with ptab before the next item refills it
}

// The item's lanes hold replicas rep_begin + 2s + 1 and + 2: a noise pair
// (2j - 1, 2j) when rep_begin is even (the planner splits paired-layout
// replicas at even offsets), unless every replica draws the parent's noise.
// The condition is the same for every lane of the warp.
template <int L, bool TAB, bool CONF = false>
__device__ __forceinline__ void run_pair_item(const ItemDev& it, const StepParams& p, float* wsm,
                                              uint4* ptab)
{
    const bool shared = (it.rep_begin & 1) == 0 && (p.flags & BD_FLAG_IDENTICAL_NOISE) == 0;
    if (shared)
        run_pair_item_k<L, TAB, CONF, true>(it, p, wsm, ptab);
    else
        run_pair_item_k<L, TAB, CONF, false>(it, p, wsm, ptab);
}

}  // namespace bdra
