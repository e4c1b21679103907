// Support kernels around the hot path: state conversion (positions <->
// bonds), replica spawn, window criteria (threshold / Bell on TSF and RSF),
// deterministic event compaction, log-survival, Exp(1) thresholds and the
// noise diagnostic.
#include <cmath>

#include "bd_support.h"

namespace bdra {

namespace {

constexpr int kThreads = 256;

inline int blocks_for(int64_t n) { return (int)((n + kThreads - 1) / kThreads); }

// Exp(1) threshold of spring i, criterion q, chain c: -ln u, u from the
// Philox stream 1 counter (i, 1 << 24, q, chain_base + c).
__global__ void exp1_kernel(const ChainDev* chains, const int32_t* spring_chain, int64_t M,
                            uint32_t k0, uint32_t k1, uint32_t chain_base, double* exp1)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const int c = spring_chain[m];
    const uint32_t i = (uint32_t)(m - chains[c].spr_off);
    for (int q = 0; q < 3; ++q) {
        const uint4 x = philox4x32_10(make_uint4(i, (uint32_t)STREAM_EXP1 << 24, (uint32_t)q,
                                                 (uint32_t)c + chain_base), k0, k1);
        const double u = ((double)x.x + 0.5) * 2.3283064365386963e-10;
        exp1[q * M + m] = -log(u);
    }
}

// Parent and every replica of spring m's chain <- r_{i+1} - r_i.
template <typename T>
__global__ void set_bonds_kernel(const ChainDev* chains, const int32_t* spring_chain, int64_t M,
                                 const double* pos, T* state)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const ChainDev ch = chains[spring_chain[m]];
    const int64_t i = m - ch.spr_off;
    const int nb = ch.N - 1;
    const double* r = pos + 3 * (ch.bead_off + i);
    const T q0 = (T)(r[3] - r[0]), q1 = (T)(r[4] - r[1]), q2 = (T)(r[5] - r[2]);
    for (int s = 0; s <= ch.R; ++s) {
        T* d = state + 3 * (ch.state_off + (int64_t)s * nb + i);
        d[0] = q0; d[1] = q1; d[2] = q2;
    }
}

// Replicas 1..R of spring m's chain <- parent.
template <typename T>
__global__ void spawn_kernel(const ChainDev* chains, const int32_t* spring_chain, int64_t M,
                             T* state)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const ChainDev ch = chains[spring_chain[m]];
    const int64_t i = m - ch.spr_off;
    const int nb = ch.N - 1;
    const T* s0 = state + 3 * (ch.state_off + i);
    const T q0 = s0[0], q1 = s0[1], q2 = s0[2];
    for (int s = 1; s <= ch.R; ++s) {
        T* d = state + 3 * (ch.state_off + (int64_t)s * nb + i);
        d[0] = q0; d[1] = q1; d[2] = q2;
    }
}

// Positions of one (chain, slot) in its centre-of-mass frame: r_0 = 0,
// r_{i+1} = r_i + Q_i (float64), minus the mean.
template <typename T>
__global__ void positions_kernel(const ChainDev* chains, const int64_t* pair_off, int n_chains,
                                 int64_t n_pairs, int all_slots, const T* state, double* out)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_pairs) return;
    int lo = 0, hi = n_chains - 1;          // chain c with pair_off[c] <= g < pair_off[c+1]
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pair_off[mid] <= g) lo = mid; else hi = mid - 1;
    }
    const ChainDev ch = chains[lo];
    const int s = (int)(g - pair_off[lo]);
    const int N = ch.N, nb = N - 1;
    const T* q = state + 3 * (ch.state_off + (int64_t)s * nb);
    double* r = out + 3 * (all_slots ? ch.slot_bead_off + (int64_t)s * N : ch.bead_off);
    double x = 0, y = 0, z = 0, sx = 0, sy = 0, sz = 0;
    for (int i = 0; i < N; ++i) {
        r[3 * i + 0] = x; r[3 * i + 1] = y; r[3 * i + 2] = z;
        sx += x; sy += y; sz += z;
        if (i < nb) { x += (double)q[3 * i]; y += (double)q[3 * i + 1]; z += (double)q[3 * i + 2]; }
    }
    sx /= N; sy /= N; sz /= N;
    for (int i = 0; i < N; ++i) { r[3 * i] -= sx; r[3 * i + 1] -= sy; r[3 * i + 2] -= sz; }
}

// RSF of window w, spring i of a chain: the chain's per-group partial sums
// (ring slot w % ring) in group order, over R.
__device__ __forceinline__ double rsf_of(const ChainDev& ch, const double* part, int64_t part_stride,
                                         int64_t slot, int64_t i)
{
    const int nb = ch.N - 1;
    const double* row = part + slot * part_stride + ch.part_off + i;
    double acc = 0.0;
    for (int g = 0; g < ch.n_groups; ++g) acc += row[(int64_t)g * nb];
    return acc / (double)ch.R;
}

// One thread per (window, spring) for the RSF and, with the conformation
// diagnostics, per (window, bead) for the per-bead Eq. 5 difference:
// dbead[w][bead][c] = (sum over the chain's groups, in group order) / R.
__global__ void rsf_fold_kernel(const FoldParams f)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per = f.M + f.NB;
    if (e >= (f.w1 - f.w0) * per) return;
    const int64_t r = e / per, x = e - r * per, w = f.w0 + r;
    if (x < f.M) {
        const ChainDev ch = f.chains[f.spring_chain[x]];
        f.rsf[w * f.M + x] = rsf_of(ch, f.part, f.part_stride, w % f.ring, x - ch.spr_off);
        return;
    }
    const int64_t bead = x - f.M;
    const ChainDev ch = f.chains[f.bead_chain[bead]];
    const int64_t i = bead - ch.bead_off;
    const double* row = f.dpart + ((w % f.ring) * f.bpart_stride + ch.bpart_off + i) * 3;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int g = 0; g < ch.n_groups; ++g) {
        const double* e3 = row + (int64_t)g * ch.N * 3;
        s0 += e3[0]; s1 += e3[1]; s2 += e3[2];
    }
    double* out = f.dbead + (w * f.NB + bead) * 3;
    out[0] = s0 / (double)ch.R; out[1] = s1 / (double)ch.R; out[2] = s2 / (double)ch.R;
}

// Threshold and Bell criteria on the window profiles TSF and RSF of windows
// [w0, w1): the force of window w is held over its S steps and the event is
// dated at the window end (w + 1) S.
__global__ void window_criteria_kernel(const ChainDev* chains, const int32_t* spring_chain,
                                       int64_t M, const double* rsf_hist, const double* tsf_hist, int64_t w0, int64_t w1, int S,
                                       double dt, int thr_mask, int bell_mask, const double* exp1,
                                       double* lam, int64_t* first_thr, int64_t* first_bell)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const ChainDev ch = chains[spring_chain[m]];
    const int64_t i = m - ch.spr_off;
    if (ch.spring == BD_SPRING_VWF && (i & 1)) return;   // disulfide bonds do not unfold
    const double dT = (double)S * dt;
    for (int q = CRIT_Q_TSF; q <= CRIT_Q_RSF; ++q) {
        const bool thr = (thr_mask >> q) & 1, bell = (bell_mask >> q) & 1;
        if (!thr && !bell) continue;
        double L = lam[q * M + m];
        int64_t ft = first_thr[q * M + m], fb = first_bell[q * M + m];
        const double E = exp1[q * M + m];
        for (int64_t w = w0; w < w1; ++w) {
            const double f = (q == CRIT_Q_RSF) ? rsf_hist[w * M + m] : tsf_hist[w * M + m];
            const int64_t step = (w + 1) * (int64_t)S;
            if (thr && ft < 0 && f >= ch.f_c) ft = step;
            if (bell) {
                L += ch.k0 * exp(f * ch.dx) * dT;
                if (fb < 0 && L >= E) fb = step;
            }
        }
        lam[q * M + m] = L;
        first_thr[q * M + m] = ft;
        first_bell[q * M + m] = fb;
    }
}

// Seed of the adjoint: dObjective / dRSF for windows w_lo .. w_lo + n_w - 1,
// G[w - w_lo][m] = grad_rsf[w - w_lo][m] (if given) plus, for the Bell
// log-survival of the RSF criterion, log S_c = -sum_w sum_i k0 exp(RSF dx) S dt
// (Sec. III), the term grad_log_surv[c] * (-k0 dx exp(RSF dx) S dt).
__global__ void adj_seed_kernel(const ChainDev* chains, const int32_t* spring_chain, int64_t M,
                                const double* rsf_hist, int64_t w_lo, int64_t n_w, const double* grad_rsf, const double* grad_log_surv,
                                int S, double dt, double* G)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_w * M) return;
    const int64_t r = e / M, m = e - r * M;
    double g = grad_rsf ? grad_rsf[e] : 0.0;
    if (grad_log_surv) {
        const int c = spring_chain[m];
        const double gl = grad_log_surv[c];
        if (gl != 0.0) {
            const ChainDev ch = chains[c];
            const double f = rsf_hist[(w_lo + r) * M + m];
            g -= gl * ch.k0 * ch.dx * exp(f * ch.dx) * ((double)S * dt);
        }
    }
    G[e] = g;
}

__device__ __forceinline__ int events_of(int64_t m, int64_t M, const int64_t* first_thr,
                                         const int64_t* first_bell)
{
    int n = 0;
    for (int q = 0; q < 3; ++q) n += (first_thr[q * M + m] >= 0) + (first_bell[q * M + m] >= 0);
    return n;
}

__device__ __forceinline__ int block_exclusive_scan(int v, int* total)
{
    __shared__ int warp_sums[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int s = lane < kThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kThreads / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    const int before = (warp > 0 ? warp_sums[warp - 1] : 0) + x - v;
    *total = warp_sums[kThreads / 32 - 1];
    __syncthreads();
    return before;
}

__global__ void event_count_kernel(int64_t M, const int64_t* first_thr, const int64_t* first_bell,
                                   int64_t* block_counts)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int v = m < M ? events_of(m, M, first_thr, first_bell) : 0;
    int total;
    block_exclusive_scan(v, &total);
    if (threadIdx.x == 0) block_counts[blockIdx.x] = total;
}

// In-place exclusive scan of n block counts; block_counts[n] <- total.
__global__ void event_scan_kernel(int64_t* block_counts, int n)
{
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += kThreads) {
        const int j = base + threadIdx.x;
        const int64_t v = j < n ? block_counts[j] : 0;
        int total;
        // counts per block fit in int (at most 6 * kThreads)
        const int before = block_exclusive_scan((int)v, &total);
        if (j < n) block_counts[j] = carry + before;
        __syncthreads();
        if (threadIdx.x == 0) carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) block_counts[n] = carry;
}

__global__ void event_write_kernel(const ChainDev* chains, const int32_t* spring_chain, int64_t M,
                                   const int64_t* first_thr, const int64_t* first_bell,
                                   const int64_t* block_offsets, bd_event* out, int64_t capacity)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int v = m < M ? events_of(m, M, first_thr, first_bell) : 0;
    int total;
    const int before = block_exclusive_scan(v, &total);
    if (m >= M || v == 0) return;
    int64_t pos = block_offsets[blockIdx.x] + before;
    const int c = spring_chain[m];
    const int32_t i = (int32_t)(m - chains[c].spr_off);
    for (int q = 0; q < 3; ++q) {
        for (int kind = 0; kind < 2; ++kind) {
            const int64_t st = kind == 0 ? first_thr[q * M + m] : first_bell[q * M + m];
            if (st < 0) continue;
            if (pos < capacity) {
                bd_event e;
                e.chain = c; e.spring = i; e.criterion = q; e.kind = kind; e.step = st;
                out[pos] = e;
            }
            ++pos;
        }
    }
}

__global__ void log_survival_kernel(const ChainDev* chains, int n_chains, int64_t M,
                                    const double* lam, double* out)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= 3 * n_chains) return;
    const int c = g / 3, q = g - 3 * (g / 3);
    const ChainDev ch = chains[c];
    double s = 0.0;
    for (int i = 0; i < ch.N - 1; ++i) s += lam[q * M + ch.spr_off + i];
    out[3 * c + q] = -s;
}

template <typename T, bool FAST>
__global__ void normals_kernel(int64_t n, const uint32_t* ctr, StepParams p, double* out)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    // the test's counter names the slot (word 1 = slot | stream << 24); the
    // generator is called with the slot's noise word
    const uint32_t slot = ctr[4 * j + 1] & 0xFFFFFFu, stream = ctr[4 * j + 1] >> 24;
    const uint4 c = make_uint4(ctr[4 * j], ((slot + 1u) >> 1) | (stream << 24), ctr[4 * j + 2],
                               ctr[4 * j + 3]);
    const uint4 x = philox4x32_10_rk(c, p.rk0, p.rk1);
    T z0, z1, z2;
    Normals<T, FAST>::draw(x, noise_half(slot), z0, z1, z2);
    const T sg = Normals<T, FAST>::sign;      // undo the fast path's sign flip
    out[3 * j] = (double)(sg * z0); out[3 * j + 1] = (double)(sg * z1); out[3 * j + 2] = (double)(sg * z2);
}

}  // namespace

cudaError_t run_exp1(const ChainDev* chains, const int32_t* spring_chain, int64_t M, uint32_t k0,
                     uint32_t k1, uint32_t chain_base, double* exp1, cudaStream_t st)
{
    if (M == 0) return cudaSuccess;
    exp1_kernel<<<blocks_for(M), kThreads, 0, st>>>(chains, spring_chain, M, k0, k1, chain_base, exp1);
    return cudaGetLastError();
}

cudaError_t run_set_bonds(bool f64, const ChainDev* chains, const int32_t* spring_chain, int64_t M,
                          const double* pos, void* state, cudaStream_t st)
{
    if (M == 0) return cudaSuccess;
    if (f64) set_bonds_kernel<double><<<blocks_for(M), kThreads, 0, st>>>(chains, spring_chain, M, pos, (double*)state);
    else set_bonds_kernel<float><<<blocks_for(M), kThreads, 0, st>>>(chains, spring_chain, M, pos, (float*)state);
    return cudaGetLastError();
}

cudaError_t run_spawn(bool f64, const ChainDev* chains, const int32_t* spring_chain, int64_t M,
                      void* state, cudaStream_t st)
{
    if (M == 0) return cudaSuccess;
    if (f64) spawn_kernel<double><<<blocks_for(M), kThreads, 0, st>>>(chains, spring_chain, M, (double*)state);
    else spawn_kernel<float><<<blocks_for(M), kThreads, 0, st>>>(chains, spring_chain, M, (float*)state);
    return cudaGetLastError();
}

cudaError_t run_positions(bool f64, const ChainDev* chains, const int64_t* pair_off, int n_chains,
                          int64_t n_pairs, int all_slots, const void* state, double* out,
                          cudaStream_t st)
{
    if (n_pairs == 0) return cudaSuccess;
    if (f64)
        positions_kernel<double><<<blocks_for(n_pairs), kThreads, 0, st>>>(
            chains, pair_off, n_chains, n_pairs, all_slots, (const double*)state, out);
    else
        positions_kernel<float><<<blocks_for(n_pairs), kThreads, 0, st>>>(
            chains, pair_off, n_chains, n_pairs, all_slots, (const float*)state, out);
    return cudaGetLastError();
}

const void* rsf_fold_func() { return (const void*)rsf_fold_kernel; }
int rsf_fold_threads() { return kThreads; }

cudaError_t run_window_criteria(const ChainDev* chains, const int32_t* spring_chain, int64_t M,
                                const double* rsf_hist, const double* tsf_hist, int64_t w0, int64_t w1, int S, double dt,
                                int thr_mask, int bell_mask, const double* exp1, double* lam,
                                int64_t* first_thr, int64_t* first_bell, cudaStream_t st)
{
    if (M == 0 || w1 <= w0) return cudaSuccess;
    window_criteria_kernel<<<blocks_for(M), kThreads, 0, st>>>(
        chains, spring_chain, M, rsf_hist, tsf_hist, w0, w1, S, dt, thr_mask,
        bell_mask, exp1, lam, first_thr, first_bell);
    return cudaGetLastError();
}

int64_t event_blocks(int64_t M) { return (M + kThreads - 1) / kThreads; }

cudaError_t run_events(const ChainDev* chains, const int32_t* spring_chain, int64_t M,
                       const int64_t* first_thr, const int64_t* first_bell, int64_t* block_scratch,
                       bd_event* out, int64_t capacity, cudaStream_t st)
{
    const int nb = (int)event_blocks(M);
    if (nb == 0) return cudaMemsetAsync(block_scratch, 0, sizeof(int64_t), st);
    event_count_kernel<<<nb, kThreads, 0, st>>>(M, first_thr, first_bell, block_scratch);
    event_scan_kernel<<<1, kThreads, 0, st>>>(block_scratch, nb);
    event_write_kernel<<<nb, kThreads, 0, st>>>(chains, spring_chain, M, first_thr, first_bell,
                                                block_scratch, out, capacity);
    return cudaGetLastError();
}

cudaError_t run_adj_seed(const ChainDev* chains, const int32_t* spring_chain, int64_t M,
                         const double* rsf_hist, int64_t w_lo, int64_t n_w,
                         const double* grad_rsf, const double* grad_log_surv, int S, double dt,
                         double* G, cudaStream_t st)
{
    adj_seed_kernel<<<blocks_for(n_w * M), kThreads, 0, st>>>(
        chains, spring_chain, M, rsf_hist, w_lo, n_w, grad_rsf, grad_log_surv, S, dt, G);
    return cudaGetLastError();
}

cudaError_t run_log_survival(const ChainDev* chains, int n_chains, int64_t M, const double* lam,
                             double* out, cudaStream_t st)
{
    log_survival_kernel<<<blocks_for(3 * (int64_t)n_chains), kThreads, 0, st>>>(chains, n_chains, M, lam, out);
    return cudaGetLastError();
}

cudaError_t run_normals(bool f64, int64_t n, const uint32_t* ctr, const StepParams& p, double* out,
                        cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    if (f64) normals_kernel<double, false><<<blocks_for(n), kThreads, 0, st>>>(n, ctr, p, out);
    else normals_kernel<float, true><<<blocks_for(n), kThreads, 0, st>>>(n, ctr, p, out);
    return cudaGetLastError();
}

}  // namespace bdra
