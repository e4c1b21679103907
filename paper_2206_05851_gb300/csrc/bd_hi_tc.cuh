// Float32 steps with hydrodynamic interaction (Eqs. 1-3) whose Cholesky
// factorisation of the Rotne-Prager-Yamakawa tensor W runs its trailing
// updates on the tensor cores.
//
// One CTA of 160 threads integrates one slot of a chain of N <= 50 beads
// (n = 3N <= 150 rows of W). The last m = n - t0 <= 126 rows and columns of W
// (t0 = 3 max(0, N - 42), a bead boundary) form the trailing block T, held in
// tensor memory (TMEM): thread i of warps 0-3 owns row i of T, TMEM lane i.
// The first t0 <= 24 rows (the head) belong to the lanes of warp 4. Per step:
//   - bead forces and normals (as the CUDA-core kernel), and the pair
//     coefficients of W (Eq. 3) once per bead pair into shared memory;
//   - every thread builds its own row of W (Eqs. 2-3, bead by bead), takes
//     the mobility-weighted force u = (W F)_row, keeps the head columns in
//     registers and stores the T columns to its TMEM lane;
//   - head: warp 4 factors the head block (one row a lane; each column's
//     root broadcast by one shuffle, its entries through shared memory); the
//     T rows solve their head columns against it (X L^T = W_T,head) and
//     T <- T - X X^T on the tensor cores;
//   - panels of 32 columns of T: warp p factors the diagonal block of
//     panel p (its 32 rows), the rows below solve against it, and the
//     tensor cores subtract the panel's outer product from the rest of T;
//     that update is issued as the next panel's 32 columns first and the
//     remaining columns after, so the next panel's factor starts as soon as
//     its own columns are done;
//   - the correlated noise w = L xi accumulates row by row as the factor's
//     entries appear; then the update and the centre-of-mass shift.
// The MMAs are kind::tf32 with float32 accumulators in TMEM, every product
// of float32 values split as hi hi + hi lo + lo hi (tf32 high parts and
// remainders), which keeps the float32 accuracy of the factor. Completion is
// tracked by two mbarriers whose waits give up after a bounded number of
// polls: the CTA then records BD_DEV_ERR_TC_WAIT, stops integrating, waits
// (bounded) for its MMAs and frees its TMEM.
#pragma once

#include "bd_hi.cuh"
#include "bd_tc.cuh"

namespace bdra {

constexpr int kTCThreads = 160;          // four row warps (TMEM lanes 0-127) + the head warp
constexpr int kTCMaxBeads = kHISmallBeads;
constexpr int kTCHeadBeads = 8;          // head of at most 24 rows
constexpr uint32_t kTCCols = 128;        // TMEM columns of a CTA
constexpr int kTCBlocksPerSM = 3;        // CTAs an SM holds (128 registers a thread; TMEM would allow 4)
static_assert(kTCBlocksPerSM * kTCCols <= 512, "TMEM columns of the resident CTAs");
constexpr uint32_t kTCPolls = 1u << 20;  // polls of a completion barrier before giving up
static_assert(3 * (kTCMaxBeads - 42) <= 3 * kTCHeadBeads, "head of the largest chain");

struct HITCShared {
    alignas(128) float op_hi[128 * 32];  // the panel's factor rows (tf32 high parts), MMA operand layout
    alignas(128) float op_lo[128 * 32];  // their remainders
    alignas(16) float4 pe[kTCMaxBeads * (kTCMaxBeads - 1) / 2];   // bead pairs bi > bj: (sqrt(c_d) d, c_i)
    alignas(16) float lt[32][32];        // factor of the current diagonal block, transposed: lt[k][j] = L[j][k]
    alignas(16) float col[2][32];        // column k of the block being factored (two in flight)
    alignas(16) float dinv[32];          // reciprocals of its diagonal
    alignas(16) float pos[4 * kHINTSmall];   // bead positions [3N] (COM frame)
    alignas(16) float frc[4 * kHINTSmall];   // bead forces [3N]
    alignas(16) float xi[4 * kHINTSmall];    // bead normals [3N]
    float com[3];
    uint16_t pr[kTCMaxBeads * (kTCMaxBeads - 1) / 2];   // pair p as (bi << 8) | bj, p = bi (bi - 1) / 2 + bj
    uint32_t taddr;                      // TMEM address of the CTA's columns
    alignas(8) uint64_t bar_next;        // MMAs of the next panel's columns done
    alignas(8) uint64_t bar_rest;        // every MMA issued so far done
};

// Per-thread bookkeeping of the CTA's tensor-memory state. Only thread 0
// (which issues the MMAs) waits on the completion barriers and tracks their
// phases; a CTA barrier then passes the completion on to the other threads.
struct TCState {
    uint32_t taddr;      // this warp's lanes (row warps), first column
    uint32_t ph_next, ph_rest;
    bool pend_next, pend_rest;
    bool bad;            // a wait gave up
    bool stall;          // BD_FLAG_TEST_TC_STALL: no MMA and no completion is issued
    int t0, m, hb, P;    // head rows, T rows, head beads, panels

    __device__ __forceinline__ void setup(int N)
    {
        const int n = 3 * N;
        hb = N > 42 ? N - 42 : 0;
        t0 = 3 * hb;
        m = n - t0;
        P = (m + 31) >> 5;
        ph_next = ph_rest = 0;
        pend_next = pend_rest = false;
        bad = false;
    }
    __device__ __forceinline__ void wait_next(HITCShared& sm)
    {
        if (threadIdx.x != 0 || !pend_next) return;
        if (!tc::mbar_wait(&sm.bar_next, ph_next, kTCPolls)) bad = true;
        ph_next ^= 1u;
        pend_next = false;
    }
    __device__ __forceinline__ void wait_rest(HITCShared& sm)
    {
        if (threadIdx.x != 0 || !pend_rest) return;
        if (!tc::mbar_wait(&sm.bar_rest, ph_rest, kTCPolls)) bad = true;
        ph_rest ^= 1u;
        pend_rest = false;
    }
};

// Pair coefficients of W (Eq. 3) for the bead pairs bi > bj of the chain:
// W's 3 x 3 block of the pair is c_d d d^T + c_i I (d = r_bj - r_bi, c_d > 0
// in both branches of Eq. 3), stored as e = sqrt(c_d) d and c_i, so that an
// entry is e_x e_y + c_i [x = y] and the transposed entries are equal bitwise.
__device__ __forceinline__ void tc_pairs(HITCShared& sm, int N, float a)
{
    const int np = N * (N - 1) / 2;
    for (int q = threadIdx.x; q < np; q += blockDim.x) {
        const int bi = sm.pr[q] >> 8, bj = sm.pr[q] & 0xFF;
        const float dx = sm.pos[3 * bj] - sm.pos[3 * bi];
        const float dy = sm.pos[3 * bj + 1] - sm.pos[3 * bi + 1];
        const float dz = sm.pos[3 * bj + 2] - sm.pos[3 * bi + 2];
        float ci, cd;
        rpy_coef<float, true>(dx, dy, dz, a, ci, cd);
        const float sc = sqrt_approx(cd);
        sm.pe[q] = make_float4(sc * dx, sc * dy, sc * dz, ci);
    }
}

// The pair table (once per kernel).
__device__ __forceinline__ void tc_pairs_init(HITCShared& sm, int N)
{
    for (int q = threadIdx.x; q < N * (N - 1) / 2; q += blockDim.x) {
        int bi = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)q)) * 0.5f);
        while (bi * (bi - 1) / 2 > q) --bi;
        while ((bi + 1) * bi / 2 <= q) ++bi;
        sm.pr[q] = (uint16_t)((bi << 8) | (q - bi * (bi - 1) / 2));
    }
}

// Row r = 3 bi + x of W at the three columns of bead bj: W[r][3 bj + y],
// zero unless `on`. Branch-free: the diagonal block reads any pair (the
// first; N >= 2) and takes the identity by selects, and bj past the chain
// is clamped for the read.
__device__ __forceinline__ void tc_w3(const HITCShared& sm, int bi, int x, int bj, int N, bool on, float& w0,
                                      float& w1, float& w2)
{
    const int bc = bj < N ? bj : N - 1;
    const int hi = bi > bc ? bi : bc, lo = bi > bc ? bc : bi;
    const bool same = hi == lo;
    const float4 e = sm.pe[same ? 0 : hi * (hi - 1) / 2 + lo];
    const float ex = same ? 0.0f : (x == 0 ? e.x : (x == 1 ? e.y : e.z));
    const float ci = same ? 1.0f : e.w;
    w0 = on ? __fmaf_rn(ex, e.x, x == 0 ? ci : 0.0f) : 0.0f;
    w1 = on ? __fmaf_rn(ex, e.y, x == 1 ? ci : 0.0f) : 0.0f;
    w2 = on ? __fmaf_rn(ex, e.z, x == 2 ? ci : 0.0f) : 0.0f;
}

// Lower Cholesky factor of a K x K block held one row a lane (A[j], j < K;
// rows beyond the block are identity rows). Column k: lane k takes the
// reciprocal square root of its diagonal and broadcasts it, the rows below
// scale their entry, and every row subtracts the column's outer product from
// its later entries, the column read from shared memory (two buffers). Each
// lane also keeps its own diagonal entry in a register, updated with its own
// column entries, so that the next column's root waits on one shuffle only.
// Returns 1 / L[lane][lane].
template <int K>
__device__ __forceinline__ float tc_warp_chol(float (&A)[32], int lane, float (*col)[32])
{
    float own_inv = 1.0f, dg = 0.0f;
#pragma unroll
    for (int j = 0; j < K; ++j)
        if (j == lane) dg = A[j];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float il = __shfl_sync(0xffffffffu, Rsqrt<float, true>::rsqrt(dg), k);
        if (lane == k) {
            A[k] = __fmul_rn(dg, il);
            own_inv = il;
        }
        const float lk = lane > k ? __fmul_rn(A[k], il) : 0.0f;
        if (lane > k) {
            A[k] = lk;
            dg = __fmaf_rn(-lk, lk, dg);
        }
        if (k + 1 < K) {
            col[k & 1][lane] = lk;
            __syncwarp();
#pragma unroll
            for (int j4 = (k + 1) & ~3; j4 < K; j4 += 4) {
                const float4 c = *reinterpret_cast<const float4*>(&col[k & 1][j4]);
                if (j4 + 0 > k) A[j4 + 0] = __fmaf_rn(-lk, c.x, A[j4 + 0]);
                if (j4 + 1 > k) A[j4 + 1] = __fmaf_rn(-lk, c.y, A[j4 + 1]);
                if (j4 + 2 > k) A[j4 + 2] = __fmaf_rn(-lk, c.z, A[j4 + 2]);
                if (j4 + 3 > k) A[j4 + 3] = __fmaf_rn(-lk, c.w, A[j4 + 3]);
            }
        }
    }
    return own_inv;
}

// A <- A L^{-T} (forward substitution over K columns) with the factor in
// sm.lt / sm.dinv; columns whose factor rows are identity rows pass through.
template <int K>
__device__ __forceinline__ void tc_row_solve(float (&A)[32], const HITCShared& sm)
{
#pragma unroll
    for (int k = 0; k < K; ++k) {
        A[k] = __fmul_rn(A[k], sm.dinv[k]);
#pragma unroll
        for (int j4 = (k + 1) & ~3; j4 < K; j4 += 4) {
            const float4 l = *reinterpret_cast<const float4*>(&sm.lt[k][j4]);
            if (j4 + 0 > k) A[j4 + 0] = __fmaf_rn(-A[k], l.x, A[j4 + 0]);
            if (j4 + 1 > k && j4 + 1 < K) A[j4 + 1] = __fmaf_rn(-A[k], l.y, A[j4 + 1]);
            if (j4 + 2 > k && j4 + 2 < K) A[j4 + 2] = __fmaf_rn(-A[k], l.z, A[j4 + 2]);
            if (j4 + 3 > k && j4 + 3 < K) A[j4 + 3] = __fmaf_rn(-A[k], l.w, A[j4 + 3]);
        }
    }
}

// Row `row` of the MMA operand (tf32 split) from A[0 .. 4 nc).
template <int NC>
__device__ __forceinline__ void tc_put_operand(HITCShared& sm, int row, const float (&A)[32], bool zero)
{
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        float h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (zero) h[e] = l[e] = 0.0f;
            else tc::split_tf32(A[4 * c + e], h[e], l[e]);
        }
        const int o = tc::op_index(row, 4 * c, 8);
        *reinterpret_cast<float4*>(&sm.op_hi[o]) = make_float4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<float4*>(&sm.op_lo[o]) = make_float4(l[0], l[1], l[2], l[3]);
    }
}

// T[:, c0 .. c0 + N) -= X X[c0 .. c0 + N)^T over ks K steps of 8, X the
// operand rows (three tf32 products per step).
__device__ __forceinline__ void tc_issue_update(HITCShared& sm, uint32_t tbase, int c0, int N, int ks)
{
    const uint32_t id = tc::idesc_tf32(128, N, true);
    const uint32_t hi = tc::smem_u32(sm.op_hi), lo = tc::smem_u32(sm.op_lo);
    const uint32_t boff = (uint32_t)(c0 >> 3) * 1024u;
#pragma unroll 1
    for (int s = 0; s < ks; ++s) {
        const uint32_t ko = 256u * (uint32_t)s;
        const uint64_t ah = tc::smem_desc(hi + ko, 128, 1024), al = tc::smem_desc(lo + ko, 128, 1024);
        const uint64_t bh = tc::smem_desc(hi + boff + ko, 128, 1024), bl = tc::smem_desc(lo + boff + ko, 128, 1024);
        tc::mma_tf32(tbase + (uint32_t)c0, ah, bh, id, true);
        tc::mma_tf32(tbase + (uint32_t)c0, ah, bl, id, true);
        tc::mma_tf32(tbase + (uint32_t)c0, al, bh, id, true);
    }
}

// The two-part update after a panel (or the head): next panel's columns
// [c1, c1 + 32), then the rest up to the padded width of T. Thread 0 only.
// With `stall` (a failure test) nothing is issued, so the waits give up.
__device__ __forceinline__ void tc_issue_two(HITCShared& sm, uint32_t tbase, int c1, int m, int ks, bool stall)
{
    if (stall) return;
    tc::fence_after_sync();
    tc_issue_update(sm, tbase, c1, 32, ks);
    tc::mma_commit(&sm.bar_next);
    const int width = (m + 15) & ~15;
    if (c1 + 32 < width) tc_issue_update(sm, tbase, c1 + 32, width - c1 - 32, ks);
    tc::mma_commit(&sm.bar_rest);
}

__device__ __forceinline__ void tc_sync()
{
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

// One step t -> t + 1 of the CTA's slot (float32). Returns the thread's
// FENE floor count; ts.bad is set (on every thread) if a wait gave up.
__device__ __forceinline__ int hi_tc_step(HITCShared& sm, TCState& ts, const ChainDev& ch,
                                          const StepConst<float, true>& k, const LJConst<float>& kl,
                                          const StepParams& p, int N,
                                          uint32_t slot_key, uint32_t chain, uint32_t step, bool harmonic, bool lj)
{
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int t0 = ts.t0, m = ts.m, hb = ts.hb, P = ts.P;
    const int floored = hi_forces<float, true>(sm, N, k, kl, harmonic, lj);
    tc_pairs(sm, N, (float)ch.hi_a);
    if (tid < N) {
        float z0, z1, z2;
        bead_noise<float, true>((uint32_t)tid, slot_key, step, chain, p, z0, z1, z2);
        sm.xi[3 * tid] = z0;
        sm.xi[3 * tid + 1] = z1;
        sm.xi[3 * tid + 2] = z2;
    }
    __syncthreads();

    // rows of W: T rows (warps 0-3) into TMEM, then their head columns into
    // registers; head rows (warp 4): the head block into registers, the rest
    // of the row for u only
    const bool head = warp == 4;
    const int row = head ? lane : t0 + tid;
    const bool valid = head ? lane < t0 : tid < m;
    const int bi = valid ? row / 3 : 0, x = valid ? row - 3 * (row / 3) : 0;
    float A[32];
    float w = 0.0f;
    float u0 = 0.0f, u1 = 0.0f, u2 = 0.0f;     // (W F)_row over the columns of each component
    if (!head) {
#pragma unroll 1
        for (int q = 0; q < 6; ++q) {         // TMEM columns [24 q, 24 q + 24): beads hb + 8 q ..
            float V[24];
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const int bj = hb + 8 * q + b;
                float w0, w1, w2;
                tc_w3(sm, bi, x, bj, N, valid && bj < N, w0, w1, w2);
                const int fb = 3 * (bj < N ? bj : N - 1);
                u0 = __fmaf_rn(w0, sm.frc[fb], u0);
                u1 = __fmaf_rn(w1, sm.frc[fb + 1], u1);
                u2 = __fmaf_rn(w2, sm.frc[fb + 2], u2);
                V[3 * b] = w0; V[3 * b + 1] = w1; V[3 * b + 2] = w2;
            }
            tc::tmem_st8(ts.taddr + 24 * q, V);
            if (q < 5) {
                tc::tmem_st8(ts.taddr + 24 * q + 8, V + 8);
                tc::tmem_st8(ts.taddr + 24 * q + 16, V + 16);
            }
        }
    } else if (valid) {
#pragma unroll 4
        for (int bj = hb; bj < N; ++bj) {
            float w0, w1, w2;
            tc_w3(sm, bi, x, bj, N, true, w0, w1, w2);
            u0 = __fmaf_rn(w0, sm.frc[3 * bj], u0);
            u1 = __fmaf_rn(w1, sm.frc[3 * bj + 1], u1);
            u2 = __fmaf_rn(w2, sm.frc[3 * bj + 2], u2);
        }
    }
#pragma unroll
    for (int b = 0; b < kTCHeadBeads; ++b) {
        float w0, w1, w2;
        tc_w3(sm, bi, x, b, N, valid && b < hb, w0, w1, w2);
        const int fb = 3 * (b < N ? b : N - 1);
        u0 = __fmaf_rn(w0, sm.frc[fb], u0);
        u1 = __fmaf_rn(w1, sm.frc[fb + 1], u1);
        u2 = __fmaf_rn(w2, sm.frc[fb + 2], u2);
        A[3 * b] = w0; A[3 * b + 1] = w1; A[3 * b + 2] = w2;
    }
    const float u = __fadd_rn(__fadd_rn(u0, u1), u2);
#pragma unroll
    for (int j = 3 * kTCHeadBeads; j < 32; ++j) A[j] = 0.0f;
    if (head && !valid) {        // identity rows below the head block
#pragma unroll
        for (int j = 0; j < 32; ++j) A[j] = j == lane ? 1.0f : 0.0f;
    }
    if (!head) tc::tmem_wait_st();
    tc_sync();

    // head: factor (warp 4), solve of the T rows, T -= X X^T
    if (t0 > 0) {
        if (head) {
            const float il = tc_warp_chol<3 * kTCHeadBeads>(A, lane, sm.col);
#pragma unroll
            for (int j = 0; j < 3 * kTCHeadBeads; ++j) sm.lt[j][lane] = A[j];
            sm.dinv[lane] = il;
            if (valid)
#pragma unroll
                for (int j = 0; j < 3 * kTCHeadBeads; ++j)
                    if (j <= lane) w = __fmaf_rn(A[j], sm.xi[j], w);
        }
        __syncthreads();
        if (!head) {
            tc_row_solve<3 * kTCHeadBeads>(A, sm);
#pragma unroll
            for (int j = 0; j < 3 * kTCHeadBeads; ++j) w = __fmaf_rn(A[j], sm.xi[j], w);
            tc_put_operand<2 * kTCHeadBeads * 3 / 8>(sm, tid, A, !valid);
        }
        tc::fence_async_smem();
        __syncthreads();
        if (tid == 0) tc_issue_two(sm, ts.taddr, 0, m, (t0 + 7) >> 3, ts.stall);
        ts.pend_next = ts.pend_rest = true;
    }

    // panels of T
#pragma unroll 1
    for (int pn = 0; pn < P; ++pn) {
        const int c0 = 32 * pn;
        ts.wait_next(sm);
        tc_sync();                 // the next panel's columns are in TMEM
        if (!head) {
            if (warp >= pn) {
                tc::tmem_ld32(ts.taddr + (uint32_t)c0, A);
                if (!valid) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) A[j] = c0 + j == tid ? 1.0f : 0.0f;
                }
            }
            if (warp == pn) {
                const float il = tc_warp_chol<32>(A, lane, sm.col);
#pragma unroll
                for (int j = 0; j < 32; ++j) sm.lt[j][lane] = A[j];
                sm.dinv[lane] = il;
                if (valid)
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (j <= lane) w = __fmaf_rn(A[j], sm.xi[t0 + c0 + j], w);
            }
        }
        ts.wait_rest(sm);          // the previous update no longer reads the operand
        tc_sync();
        if (!head && warp > pn) {
            tc_row_solve<32>(A, sm);
            if (valid)
#pragma unroll
                for (int j = 0; j < 32; ++j) w = __fmaf_rn(A[j], sm.xi[t0 + c0 + j], w);
        }
        if (pn + 1 < P) {
            if (!head && warp > pn) tc_put_operand<8>(sm, tid, A, !valid);
            tc::fence_async_smem();
            __syncthreads();
            if (tid == 0) tc_issue_two(sm, ts.taddr, c0 + 32, m, 4, ts.stall);
            ts.pend_next = ts.pend_rest = true;
        } else {
            __syncthreads();       // every read of sm.lt done before the next step writes it
        }
    }
    ts.wait_next(sm);
    ts.wait_rest(sm);
    tc::fence_before_sync();
    ts.bad = __syncthreads_or(ts.bad) != 0;    // every MMA of the step is done
    tc::fence_after_sync();

    // update and centre-of-mass shift
    float nv = 0.0f;
    if (valid) {
        const int xx = row % 3, b3 = row - xx;
        const float r = sm.pos[row];
        const float fl = xx == 0 ? fmaf(k.axz, sm.pos[b3 + 2], fmaf(k.axx, r, r))
                                 : (xx == 1 ? fmaf(k.ayy, r, r) : fmaf(k.azz, r, r));
        nv = fmaf(k.cn, w, fmaf(k.cd, u, fl));
    }
    __syncthreads();
    if (valid) sm.pos[row] = nv;
    __syncthreads();
    if (tid < 32) {
        float s[3] = {0.0f, 0.0f, 0.0f};
        for (int b = tid; b < N; b += 32)
#pragma unroll
            for (int c = 0; c < 3; ++c) s[c] += sm.pos[3 * b + c];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s[c] += __shfl_xor_sync(0xffffffffu, s[c], o);
        }
        if (tid == 0)
#pragma unroll
            for (int c = 0; c < 3; ++c) sm.com[c] = s[c] / (float)N;
    }
    __syncthreads();
    if (tid < 3 * N) sm.pos[tid] -= sm.com[tid % 3];
    __syncthreads();
    return floored;
}

// Set-up of a CTA: barriers and TMEM columns (warp 0); every thread's state.
__device__ __forceinline__ void hi_tc_begin(HITCShared& sm, TCState& ts, int N)
{
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        tc::mbar_init(&sm.bar_next, 1);
        tc::mbar_init(&sm.bar_rest, 1);
    }
    for (int e = threadIdx.x; e < 128 * 32; e += blockDim.x) sm.op_hi[e] = sm.op_lo[e] = 0.0f;
    tc_pairs_init(sm, N);
    if (warp == 0) {
        tc::tmem_alloc(&sm.taddr, kTCCols);
        tc::tmem_relinquish();
    }
    tc_sync();
    ts.setup(N);
    ts.taddr = sm.taddr + ((uint32_t)(32 * (warp & 3)) << 16);
}

// End of a CTA: MMAs still in flight (after a wait that gave up) are waited
// for once more, bounded, then the TMEM columns are freed.
__device__ __forceinline__ void hi_tc_end(HITCShared& sm, TCState& ts, int32_t* dev_err)
{
    ts.wait_next(sm);
    ts.wait_rest(sm);
    const bool bad = __syncthreads_or(ts.bad) != 0;
    if (bad && threadIdx.x == 0) atomicOr(dev_err, BD_DEV_ERR_TC_WAIT);
    tc_sync();
    if ((threadIdx.x >> 5) == 0) tc::tmem_dealloc(sm.taddr, kTCCols);
}

// The tensor-core engine of a slot (the kernel bodies of bd_hi.cuh).
struct HITCEngine {
    using Shared = HITCShared;
    TCState ts;
    __device__ __forceinline__ void begin(Shared& sm, int N, int32_t flags)
    {
        for (int e = threadIdx.x; e < 4 * kHINTSmall; e += blockDim.x) {
            sm.pos[e] = 0.0f; sm.frc[e] = 0.0f; sm.xi[e] = 0.0f;
        }
        hi_tc_begin(sm, ts, N);
        ts.stall = (flags & BD_FLAG_TEST_TC_STALL) != 0;
    }
    __device__ __forceinline__ int step(Shared& sm, const ChainDev& ch, const StepConst<float, true>& k,
                                        const LJConst<float>& kl, const StepParams& p, int N, uint32_t key,
                                        uint32_t chain, uint32_t t, bool harmonic, bool lj)
    {
        return hi_tc_step(sm, ts, ch, k, kl, p, N, key, chain, t, harmonic, lj);
    }
    __device__ __forceinline__ bool failed() const { return ts.bad; }
    __device__ __forceinline__ void end(Shared& sm, int32_t* dev_err) { hi_tc_end(sm, ts, dev_err); }
};

__global__ void __launch_bounds__(kTCThreads, kTCBlocksPerSM) hi_tc_replica_kernel(const StepParams p)
{
    extern __shared__ __align__(128) unsigned char hi_tc_smem_raw[];
    hi_replica_body<float, true, HITCEngine>(p, *reinterpret_cast<HITCShared*>(hi_tc_smem_raw));
}

__global__ void __launch_bounds__(kTCThreads, kTCBlocksPerSM) hi_tc_parent_kernel(const StepParams p)
{
    extern __shared__ __align__(128) unsigned char hi_tc_smem_raw[];
    hi_parent_body<float, true, HITCEngine>(p, *reinterpret_cast<HITCShared*>(hi_tc_smem_raw));
}

}  // namespace bdra
