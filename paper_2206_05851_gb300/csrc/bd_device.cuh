// Device-side building blocks of the replica-averaged Brownian-dynamics path:
// the counter-based noise of Eq. 1, the spring law and the parameter blocks
// that the host hands to the kernels. Written for sm_103a.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/bdra.h"

namespace bdra {

// ---------------------------------------------------------------------------
// Parameter blocks (plain data, shared by host and device code)
// ---------------------------------------------------------------------------

// One chain, as the kernels need it. Bond vectors Q_i = r_{i+1} - r_i of
// every slot (0 = parent, 1..R = replicas) are stored slot-major:
// state[(state_off + slot * (N-1) + i) * 3 + d].
struct ChainDev {
    int32_t N, R, n_groups, spring;   // spring: BD_SPRING_* law
    int64_t bead_off;    // first bead of this chain in a [sum N][3] position array
    int64_t slot_bead_off;  // first bead in an all-slot [sum (R+1) N][3] array
    int64_t state_off;   // bond index of slot 0, bond 0
    int64_t spr_off;     // first spring of this chain in an [M] profile
    int64_t part_off;    // first entry of group 0 in a per-window partial row
    int64_t rep_off;     // replicas of the chains before this one (sum R)
    int64_t bpart_off;   // first entry of group 0 in a per-window per-bead partial row
    double H, Hinvb;     // spring constant; H/b for FENE, 0 for Hooke
    double kxx, kyy, kzz, kxz;   // velocity gradient, v = kappa . r
    double f_c, k0, dx;  // threshold force; Bell rate k0 exp(f dx)
    double r0, lj_u, lj_s2;  // harmonic rest length; Lennard-Jones depth and min distance^2
    double hi_a;         // RPY bead radius (hydrodynamic interaction); 0: free draining
    double vwf_fa, vwf_fb, vwf_ix2;  // vWF A2 domains: FENE and harmonic constants, 1 / x_max^2
    // float32 step constants, rounded once on the host from the values
    // above (so the kernels never rebuild them from doubles): H, H/b, D dt,
    // sqrt(2 D dt) times the fast normals' sign, kappa_xx dt, kappa_yy dt,
    // kappa_zz dt, kappa_xz dt, s_min
    float f32[9];
    float f32_pad;
};

// One warp's work: replicas rep_begin + 1 + stride s, s = 0 .. rep_count-1,
// of `chain` (group `group` of the chain's replica-force partial sums),
// evolved with the step variant `variant` (springs per lane, one or two
// replicas per lane; see Variant). stride 2 keeps the replicas of a
// one-replica-per-lane item all odd or all even, so that every lane of the
// warp draws the same half of its noise pair's generator output.
struct ItemDev {
    int32_t chain, group, rep_begin, rep_count;
    int32_t variant, stride;
};

// Threads of every parent-kernel CTA and of every adjoint-kernel CTA (the
// kernels size their shared tables by them).
constexpr int kParentThreads = 64;
constexpr int kAdjThreads = 128;

// One warp of the parent kernel: `count` parents, chains
// parent_items[first .. first+count-1], each on G lanes.
struct ParentWarp {
    int32_t first, count, G, pad;
};

// Step variants: one replica per lane with L springs (code L), or two
// replicas per lane with L springs (code kPairBase + L, float32 only).
constexpr int32_t kPairBase = 100;
// Collapsed-chain variants (harmonic springs with rest length, Lennard-Jones
// pair forces; one replica per lane): code kLJBase + L.
constexpr int32_t kLJBase = 200;
// Chains with hydrodynamic interaction (Eqs. 1-3): one CTA per replica.
constexpr int32_t kHIBase = 300;

// Bits of StepParams::dev_err.
enum { BD_DEV_ERR_TC_WAIT = 1 };   // a tensor-core completion wait gave up

struct StepParams {
    const ChainDev* chains;
    const ItemDev* items;       // replica kernel: warp work items, longest first
    int32_t n_items;
    int32_t* queue;             // next unclaimed work item (zeroed before each launch)
    const int32_t* parent_items;  // parent kernel: chain ids
    const ParentWarp* parent_warps;  // parent kernel: warps of this launch
    int32_t n_parent_warps;
    void* state;                // T [state_elems][3]
    void* snap;                 // T [win_ring][M][3] parent at the start of window w, row w % win_ring
    double* part_hist;          // [win_ring][part_stride] per-group replica sums, window w at w % win_ring
    double* tsf_hist;           // [max_windows][M] parent window means
    double* tsf_acc;            // [M] parent's running sum inside the current window
    double* lam;                // [3][M] integrated Bell hazard
    int64_t* first_thr;         // [3][M]
    int64_t* first_bell;        // [3][M]
    const double* exp1;         // [3][M] Exp(1) thresholds
    unsigned long long* overext;  // [n_chains]
    int32_t* dev_err;           // error bits of kernels whose bounded waits gave up (BD_DEV_ERR_*)
    // conformation diagnostics of Eq. 5 (with BD_FLAG_CONFORMATION)
    double* dbar;               // [max_windows][sum R][3] replica vs halted parent, bead mean
    double* dbead_part;         // [win_ring][bpart_stride][3] per-group per-bead sums
    double* rgz;                // [max_windows][n_chains] parent's z radius of gyration
    int64_t n_rep, bpart_stride;
    int32_t n_chains;
    uint32_t chain_base;        // noise-counter chain word of chain 0 (chain c: chain_base + c)
    int64_t part_stride, M;
    int32_t win_ring, pad_ring;  // windows one chunk touches (started or ended) + 1
    int64_t t0, n_steps;
    double dt, s_min;
    int32_t S, flags, thr_mask, bell_mask;
    uint32_t key0, key1;
    // Philox round keys (key + r * Weyl constant, r = 0..9): read straight
    // from the kernel-parameter bank instead of occupying registers.
    uint32_t rk0[10], rk1[10];
};

// Adjoint (bd_adjoint.cuh): per chain, for the adjoint only.
struct AdjChain {
    int64_t part_off;    // first entry of this chain's group 0 in a mu row
    int32_t n_groups;    // adjoint replica groups (warp items) of the chain
    int32_t pad;
    double khat[4];      // kappa / rate: xx, yy, zz, xz
};

struct AdjParams {
    StepParams sp;             // forward parameters: chains, parent warps, keys, dt, S
    const AdjChain* adj;
    const ItemDev* items;      // replica work items of this launch (one tile)
    int32_t n_items;
    int32_t n_steps;           // parent kernels: steps of this launch
    int64_t t0;                // parent kernels: first step
    const void* ckpt;          // T [n_ckpt][M][3] parent every K steps from the origin
    int64_t ckpt_index;        // checkpoint the parent recompute starts from
    void* segbuf;              // T [K + 1][M][3] parent states of the segment
    int64_t seg_t0;            // step of segbuf row 0
    void* repbuf;              // T [batch][S + 1][state_bonds][3] replica states
    int64_t state_bonds;
    int64_t w_batch0;          // replica kernel: window of blockIdx.y = 0
    void* lamP;                // T [M][3] parent adjoint carried between segments
    const double* G;           // [w_hi - w_lo][M] dObjective / dRSF, row 0 = window w_lo
    double* mu;                // [rows][mu_stride][3] window sensitivities
    int64_t mu_w0, mu_stride;
    int64_t w_lo, w_hi;        // the objective's windows: w_lo <= w < w_hi
    double* grad;              // [n_chains][3] dObjective / d(rate, b, H)
};

// Fold of the per-group partial sums of windows [w0, w1) into the RSF
// history: rsf[w][m] = (sum over the chain's groups, in group order) / R.
struct FoldParams {
    const ChainDev* chains;
    const int32_t* spring_chain;
    const double* part;          // [ring][part_stride]
    double* rsf;                 // [max_windows][M]
    int64_t M, part_stride, w0, w1;
    int32_t ring, pad;
    // per-bead conformation differences (NB = 0: none): [ring][bpart_stride][3] -> [max_windows][NB][3]
    const int32_t* bead_chain;   // [NB]
    const double* dpart;
    double* dbead;
    int64_t NB, bpart_stride;
};

enum { CRIT_Q_ISF = 0, CRIT_Q_TSF = 1, CRIT_Q_RSF = 2 };
enum { STREAM_BD = 0, STREAM_EXP1 = 1 };

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies, XOR of the high halves with the other counter words
// and the round key, and a fixed permutation; Weyl key schedule. The key is
// uniform across the grid, so the round keys fold into uniform registers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = 0xD2511F53ull * (unsigned long long)c.x;
        const unsigned long long p1 = 0xCD9E8D57ull * (unsigned long long)c.z;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Same generator with precomputed round keys rk0[r] = k0 + r W0,
// rk1[r] = k1 + r W1 (as held in StepParams).
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const uint32_t (&rk0)[10],
                                                  const uint32_t (&rk1)[10])
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = 0xD2511F53ull * (unsigned long long)c.x;
        const unsigned long long p1 = 0xCD9E8D57ull * (unsigned long long)c.z;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c = make_uint4(hi1 ^ c.y ^ rk0[r], lo1, hi0 ^ c.w ^ rk1[r], lo0);
    }
    return c;
}

// The same generator split by what the counter words depend on, for the
// integrator's counter (bead, slot word, step, chain): after two rounds the
// state is (B.x ^ S.x, B.y, S.y ^ B.z, S.z), where B depends only on (bead,
// chain) and S only on (step, slot word). B is computed once per bead and S
// once per step, so a bead-step runs rounds 3..10 only. Exact integer
// arithmetic: the output is bitwise that of philox4x32_10_rk.
// High and low words of a Philox 32 x 32 -> 64 product. BD_PHILOX_HILO
// selects two 32-bit multiplies (high, low) instead of one wide multiply.
#ifndef BD_PHILOX_HILO
#define BD_PHILOX_HILO 0
#endif
__device__ __forceinline__ void philox_mulhilo(uint32_t m, uint32_t x, uint32_t& hi, uint32_t& lo)
{
#if BD_PHILOX_HILO
    hi = __umulhi(m, x);
    lo = m * x;
#else
    const unsigned long long p = (unsigned long long)m * (unsigned long long)x;
    hi = (uint32_t)(p >> 32);
    lo = (uint32_t)p;
#endif
}

struct PhiloxSplit {
    static __device__ __forceinline__ uint4 bead_part(uint32_t bead, uint32_t chain,
                                                      const uint32_t (&rk0)[10],
                                                      const uint32_t (&rk1)[10])
    {
        const unsigned long long p0 = 0xD2511F53ull * (unsigned long long)bead;
        const uint32_t x2 = (uint32_t)(p0 >> 32) ^ chain ^ rk1[0];
        const unsigned long long p1 = 0xCD9E8D57ull * (unsigned long long)x2;
        return make_uint4((uint32_t)(p1 >> 32) ^ rk0[1], (uint32_t)p1, (uint32_t)p0 ^ rk1[1], 0u);
    }
    static __device__ __forceinline__ uint3 step_part(uint32_t step, uint32_t slot_word,
                                                      const uint32_t (&rk0)[10])
    {
        const unsigned long long p1 = 0xCD9E8D57ull * (unsigned long long)step;
        const uint32_t x0 = (uint32_t)(p1 >> 32) ^ slot_word ^ rk0[0];
        const unsigned long long p0 = 0xD2511F53ull * (unsigned long long)x0;
        return make_uint3((uint32_t)p1, (uint32_t)(p0 >> 32), (uint32_t)p0);
    }
    static __device__ __forceinline__ uint4 finish(uint4 b, uint3 s, const uint32_t (&rk0)[10],
                                                   const uint32_t (&rk1)[10])
    {
        uint4 c = make_uint4(b.x ^ s.x, b.y, s.y ^ b.z, s.z);
#pragma unroll
        for (int r = 2; r < 10; ++r) {
            uint32_t hi0, lo0, hi1, lo1;
            philox_mulhilo(0xD2511F53u, c.x, hi0, lo0);
            philox_mulhilo(0xCD9E8D57u, c.z, hi1, lo1);
            c = make_uint4(hi1 ^ c.y ^ rk0[r], lo1, hi0 ^ c.w ^ rk1[r], lo0);
        }
        return c;
    }
};

// ---------------------------------------------------------------------------
// Standard normals of a slot (the random displacement R_i of Eq. 1, three per
// bead and step). Replicas 2j-1 and 2j share one Philox output per (bead,
// step): counter word 1 is j | stream << 24 (the parent, slot 0: j = 0). The
// output's 128 bits give six 21-bit uniforms u = (m + 1/2) 2^-21: m0..m3 the
// top 21 bits of words 0..3, m4 the low 11 bits of word 0 above the low 10
// bits of word 1, m5 the same of words 2 and 3. Box-Muller turns the pairs
// (u0, u1), (u2, u3), (u4, u5) (radius uniform, angle uniform) into six
// normals z = r (cos, sin)(2 pi u_angle), r = sqrt(-2 ln u_radius); half 0
// (the odd replica slot and the parent) is (z0, z1, z2), half 1 (the even
// replica slot) is (z3, z4, z5). So a lane that holds a replica pair draws
// both replicas' noise from one generator call.
//
// Normals<T, FAST>::sign: the FAST float path returns the normals with their
// sign flipped (it evaluates cos and sin of 2 pi u - pi, the accurate range of
// the hardware units, and cos(2 pi u - pi) = -cos(2 pi u)). The step
// multiplies its noise coefficient by `sign`, which undoes the flip exactly:
// (-a) - (-b) = -(a - b) and (-c)(-d) = c d in floating point.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t noise_word(uint32_t slot)
{
    return ((slot + 1u) >> 1) | ((uint32_t)STREAM_BD << 24);
}
__device__ __forceinline__ uint32_t noise_half(uint32_t slot)
{
    return (slot != 0u && (slot & 1u) == 0u) ? 1u : 0u;
}

// The six 21-bit fields m_k of a Philox output.
struct Fields21 {
    static __device__ __forceinline__ uint32_t m(uint4 x, int k)
    {
        switch (k) {
        case 0: return x.x >> 11;
        case 1: return x.y >> 11;
        case 2: return x.z >> 11;
        case 3: return x.w >> 11;
        case 4: return ((x.x & 0x7FFu) << 10) | (x.y & 0x3FFu);
        default: return ((x.z & 0x7FFu) << 10) | (x.w & 0x3FFu);
        }
    }
    // The float 1 + m_k 2^-21 (exact: m_k fills the top 21 of the 23
    // mantissa bits), built from the words without isolating m_k first.
    static __device__ __forceinline__ float one_plus(uint4 x, int k)
    {
        const uint32_t one = 0x3F800000u;
        switch (k) {
        case 0: return __uint_as_float(one | ((x.x >> 9) & 0x7FFFFCu));
        case 1: return __uint_as_float(one | ((x.y >> 9) & 0x7FFFFCu));
        case 2: return __uint_as_float(one | ((x.z >> 9) & 0x7FFFFCu));
        case 3: return __uint_as_float(one | ((x.w >> 9) & 0x7FFFFCu));
        case 4: return __uint_as_float(((x.x << 12) & 0x7FF000u) | (((x.y << 2) & 0xFFCu) | one));
        default: return __uint_as_float(((x.z << 12) & 0x7FF000u) | (((x.w << 2) & 0xFFCu) | one));
        }
    }
};

// Per-spring window sums of a parent: the running sum of its ISF samples
// for the TSF (Sec. II) and the ISF Bell hazard of the current window with
// the Exp(1) budget left at its start, rem = E - Lambda (Sec. III; a first
// passage when the window's hazard reaches rem). Lambda itself lives in
// float64 memory and is advanced at every window end and launch end.
struct BellConst {
    double k0dt, dx;     // k0 dt and dx of the chain's Bell law
    float dxf, lnk;      // dx and ln(k0 dt) (-inf for k0 dt <= 0) in float32
    __device__ void load(double k0, double dt, double dx_)
    {
        k0dt = k0 * dt;
        dx = dx_;
        dxf = (float)dx_;
        lnk = k0dt > 0.0 ? (float)log(k0dt) : -INFINITY;
    }
};

template <typename T> struct ParentSums;

// Float64 integration: float64 sums.
template <> struct ParentSums<double> {
    double tsf, haz, rem;
    __device__ __forceinline__ void start(double tsf0, double rem0)
    {
        tsf = tsf0;
        haz = 0.0;
        rem = rem0;
    }
    __device__ __forceinline__ void add_isf(double f) { tsf += f; }
    // one step's hazard k0 dt e^(dx f); true once the window's hazard reaches rem
    __device__ __forceinline__ bool add_hazard(double f, const BellConst& b, double*)
    {
        haz = fma(b.k0dt, exp(b.dx * f), haz);
        return haz >= rem;
    }
    __device__ __forceinline__ double tsf_sum() const { return tsf; }
    __device__ __forceinline__ double hazard() const { return haz; }
    __device__ __forceinline__ void next_window(double rem0)
    {
        tsf = 0.0;
        haz = 0.0;
        rem = rem0;
    }
};

// Float32 integration. Summing the float32 samples in float64 took two or
// three float64 instructions per spring and step (widening, add, compare),
// and float64 runs at 1/64 of the float32 rate on this GPU: the parent
// kernels were float64-pipe bound. The sums are float-float pairs instead,
// value hi + lo: each addition is the error-free TwoSum followed by a
// renormalisation, so |lo| <= ulp(hi) / 2 and a sum of n terms is within
// n 2^-47 max|partial sum| of the exact one (n 2^-53 for a float64 sum):
// 1.1e-11 of the mean sample for a 1500-step window. The hazard increment
// k0 dt e^(dx f) = e^y, y = dx f + ln(k0 dt), is taken in float32 (three
// roundings in y, about 1e-6 absolute for |y| up to 20, and expf within 2
// ulp): about 1e-6 relative, an order below the error the float32 tension
// itself brings. An increment outside e^(+-64) (e^64 = 6e27, far past any
// budget; e^-64 = 2e-28, below float32's reach in a sum) takes the float64
// exponential and goes straight into Lambda in memory, the budget lowered by
// the same amount, so the pairs neither overflow nor flush tiny hazards to
// zero where the float64 sums would not.
__device__ __forceinline__ void ff_add(float& hi, float& lo, float x)
{
    const float s = __fadd_rn(hi, x);
    const float bp = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    const float l = __fadd_rn(lo, e);
    hi = __fadd_rn(s, l);
    lo = __fsub_rn(l, __fsub_rn(hi, s));
}
__device__ __forceinline__ void ff_from(double d, float& hi, float& lo)
{
    hi = __double2float_rn(d);
    lo = isinf(hi) ? 0.0f : __double2float_rn(d - (double)hi);
}
__device__ __forceinline__ double ff_to(float hi, float lo) { return (double)hi + (double)lo; }

template <> struct ParentSums<float> {
    float t_hi, t_lo, h_hi, h_lo, r_hi, r_lo;
    __device__ __forceinline__ void start(double tsf0, double rem0)
    {
        ff_from(tsf0, t_hi, t_lo);
        h_hi = h_lo = 0.0f;
        ff_from(rem0, r_hi, r_lo);
    }
    __device__ __forceinline__ void add_isf(float f) { ff_add(t_hi, t_lo, f); }
    __device__ __forceinline__ bool add_hazard(float f, const BellConst& b, double* lam)
    {
        const float y = __fadd_rn(__fmul_rn(b.dxf, f), b.lnk);
        if (fabsf(y) < 64.0f) {
            ff_add(h_hi, h_lo, expf(y));
        } else {
            const double inc = b.k0dt * exp(b.dx * (double)f);
            *lam += inc;
            ff_from(ff_to(r_hi, r_lo) - inc, r_hi, r_lo);
        }
        return __fadd_rn(__fsub_rn(h_hi, r_hi), __fsub_rn(h_lo, r_lo)) >= 0.0f;
    }
    __device__ __forceinline__ double tsf_sum() const { return ff_to(t_hi, t_lo); }
    __device__ __forceinline__ double hazard() const { return ff_to(h_hi, h_lo); }
    __device__ __forceinline__ void next_window(double rem0)
    {
        t_hi = t_lo = h_hi = h_lo = 0.0f;
        ff_from(rem0, r_hi, r_lo);
    }
};

template <typename T, bool FAST> struct Normals;

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Hardware log2 / sin / cos with denormals flushed: the Box-Muller
// arguments are never denormal (u >= 2^-22, |angle| >= 2 pi 2^-22), so the
// flush changes no result and spares the denormal handling.
__device__ __forceinline__ float lg2_approx(float x)
{
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float sin_approx(float x)
{
    float r;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float cos_approx(float x)
{
    float r;
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Building blocks of the fast float Box-Muller, shared by the one-slot and
// two-slot (packed) paths so both round identically.
struct FastBM {
    static constexpr float m2ln2 = -2.0f * 0.69314718055994531f;
    static constexpr float twopi = 6.2831853071795865f;
    // 1 - 2^-22: (1 + m 2^-21) - this = (m + 1/2) 2^-21 exactly
    static constexpr float rad_off = 0.99999976158142090f;
    // angle 2 pi (1 + m 2^-21) + off = 2 pi u - pi
    static constexpr float off = -6.2831853071795865f * (1.5f - 2.384185791015625e-7f);
    // radius r of field k (radius uniforms: k = 0, 2, 4)
    static __device__ __forceinline__ float radius(uint4 x, int k)
    {
        const float u = __fsub_rn(Fields21::one_plus(x, k), rad_off);
        // |a| guards the approximate log2 of values within an ulp of 1
        return sqrt_approx(fabsf(__fmul_rn(m2ln2, lg2_approx(u))));
    }
    // angle 2 pi u - pi of field k (angle uniforms: k = 1, 3, 5)
    static __device__ __forceinline__ float angle(uint4 x, int k)
    {
        return __fmaf_rn(Fields21::one_plus(x, k), twopi, off);
    }
};

// Box-Muller pair PR (radius field 2 PR, angle field 2 PR + 1) in float or
// double with the library's log / sqrt / sincospi: r cos (WANT 1 or 3) and
// r sin (WANT 2 or 3) of the angle; only the wanted ones are evaluated.
template <typename T, int PR, int WANT>
__device__ __forceinline__ void bm_pair(uint4 x, T& c, T& s)
{
    const T s21 = T(4.76837158203125e-7);                  // 2^-21
    const T ur = ((T)Fields21::m(x, 2 * PR) + T(0.5)) * s21;
    const T ua = ((T)Fields21::m(x, 2 * PR + 1) + T(0.5)) * s21;
    const T r = sqrt(T(-2) * log(ur));
    if (WANT == 3) {
        T sn, cs;
        sincospi(T(2) * ua, &sn, &cs);
        c = r * cs;
        s = r * sn;
    } else if (WANT == 1) {
        c = r * cospi(T(2) * ua);
    } else {
        s = r * sinpi(T(2) * ua);
    }
}

template <bool FAST> struct Normals<float, FAST> {
    static constexpr float sign = FAST ? -1.0f : 1.0f;
    // the three normals of half H (0: z0 z1 z2, 1: z3 z4 z5)
    template <int H>
    static __device__ __forceinline__ void draw_h(uint4 x, float& z0, float& z1, float& z2)
    {
        if (FAST) {
            if (H == 0) {
                const float r0 = FastBM::radius(x, 0), r2 = FastBM::radius(x, 2);
                const float t1 = FastBM::angle(x, 1), t3 = FastBM::angle(x, 3);
                z0 = __fmul_rn(r0, cos_approx(t1));
                z1 = __fmul_rn(r0, sin_approx(t1));
                z2 = __fmul_rn(r2, cos_approx(t3));
            } else {
                const float r2 = FastBM::radius(x, 2), r4 = FastBM::radius(x, 4);
                const float t3 = FastBM::angle(x, 3), t5 = FastBM::angle(x, 5);
                z0 = __fmul_rn(r2, sin_approx(t3));
                z1 = __fmul_rn(r4, cos_approx(t5));
                z2 = __fmul_rn(r4, sin_approx(t5));
            }
        } else {
            float c1 = 0.0f, s1 = 0.0f, c2 = 0.0f, s2 = 0.0f;
            if (H == 0) {
                bm_pair<float, 0, 3>(x, c1, s1);
                bm_pair<float, 1, 1>(x, c2, s2);
                z0 = c1; z1 = s1; z2 = c2;
            } else {
                bm_pair<float, 1, 2>(x, c1, s1);
                bm_pair<float, 2, 3>(x, c2, s2);
                z0 = s1; z1 = c2; z2 = s2;
            }
        }
    }
    // half h known only at run time (both forms are in the code: callers that
    // know it at compile time use draw_h)
    static __device__ __forceinline__ void draw(uint4 x, uint32_t h, float& z0, float& z1, float& z2)
    {
        if (h == 0) draw_h<0>(x, z0, z1, z2);
        else draw_h<1>(x, z0, z1, z2);
    }
};

template <bool FAST> struct Normals<double, FAST> {
    static constexpr double sign = 1.0;
    template <int H>
    static __device__ __forceinline__ void draw_h(uint4 x, double& z0, double& z1, double& z2)
    {
        double c1 = 0.0, s1 = 0.0, c2 = 0.0, s2 = 0.0;
        if (H == 0) {
            bm_pair<double, 0, 3>(x, c1, s1);
            bm_pair<double, 1, 1>(x, c2, s2);
            z0 = c1; z1 = s1; z2 = c2;
        } else {
            bm_pair<double, 1, 2>(x, c1, s1);
            bm_pair<double, 2, 3>(x, c2, s2);
            z0 = s1; z1 = c2; z2 = s2;
        }
    }
    static __device__ __forceinline__ void draw(uint4 x, uint32_t h, double& z0, double& z1, double& z2)
    {
        if (h == 0) draw_h<0>(x, z0, z1, z2);
        else draw_h<1>(x, z0, z1, z2);
    }
};

// Draw with the half fixed at compile time (H = 0, 1) or read at run time
// (H = -1: h).
template <typename T, bool FAST, int H>
__device__ __forceinline__ void draw_half(uint4 x, uint32_t h, T& z0, T& z1, T& z2)
{
    if (H == 0) Normals<T, FAST>::template draw_h<0>(x, z0, z1, z2);
    else if (H == 1) Normals<T, FAST>::template draw_h<1>(x, z0, z1, z2);
    else Normals<T, FAST>::draw(x, h, z0, z1, z2);
}

// The same normals from the split generator: bp = PhiloxSplit::bead_part of
// the bead, sp = PhiloxSplit::step_part of the step and noise word, h the
// slot's half (or H at compile time).
template <typename T, bool FAST, int H = -1>
__device__ __forceinline__ void bead_noise_split(uint4 bp, uint3 sp, const StepParams& p, uint32_t h,
                                                 T& z0, T& z1, T& z2)
{
    draw_half<T, FAST, H>(PhiloxSplit::finish(bp, sp, p.rk0, p.rk1), h, z0, z1, z2);
}

// The normals of (bead, slot, step, chain) from the full generator.
template <typename T, bool FAST, int H = -1>
__device__ __forceinline__ void bead_noise(uint32_t bead, uint32_t slot, uint32_t step,
                                           uint32_t chain, const StepParams& p,
                                           T& z0, T& z1, T& z2)
{
    const uint4 x = philox4x32_10_rk(make_uint4(bead, noise_word(slot), step, chain), p.rk0, p.rk1);
    draw_half<T, FAST, H>(x, noise_half(slot), z0, z1, z2);
}

// ---------------------------------------------------------------------------
// Spring law: F = H Q / s with s = 1 - (H/b) Q^2 (FENE, floored at s_min;
// Hooke has H/b = 0 so s = 1). Returns the coefficient H / s.
// ---------------------------------------------------------------------------
template <typename T, bool FAST> struct Div {
    static __device__ __forceinline__ T div(T a, T b) { return a / b; }
};
template <> struct Div<float, true> {
    static __device__ __forceinline__ float div(float a, float b) { return a * rcp_approx(b); }
};

template <typename T>
__device__ __forceinline__ T bond_q2(T qx, T qy, T qz)
{
    return fma(qx, qx, fma(qy, qy, qz * qz));
}

template <typename T, bool FAST>
__device__ __forceinline__ T spring_coef(T qx, T qy, T qz, T H, T Hinvb, T smin, int& floored)
{
    const T s = fma(-Hinvb, bond_q2(qx, qy, qz), T(1));
    floored += s < smin;
    return Div<T, FAST>::div(H, fmax(s, smin));
}

template <typename T, bool FAST>
__device__ __forceinline__ T spring_tension(T qx, T qy, T qz, T H, T Hinvb, T smin)
{
    int dummy = 0;
    const T c = spring_coef<T, FAST>(qx, qy, qz, H, Hinvb, smin, dummy);
    return c * sqrt(bond_q2(qx, qy, qz));
}

}  // namespace bdra
