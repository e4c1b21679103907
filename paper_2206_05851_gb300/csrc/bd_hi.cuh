// Hydrodynamic interaction (Eqs. 1-3): chains whose beads move with the
// Rotne-Prager-Yamakawa diffusion tensor. In the units of Eq. 1 used here the
// single-bead diffusivity is D_0 = 1/4 and D = D_0 W, with W_ii = I (Eq. 2)
// and, for beads i != j at separation d = r_j - r_i, r = |d| (Eq. 3 over D_0,
// a the bead radius):
//   r >= 2a:  W_ij = (3a / 4r) [(1 + 2a^2/(3r^2)) I + (1 - 2a^2/r^2) d d / r^2]
//   r <  2a:  W_ij = (1 - 9r/(32a)) I + (3r/(32a)) d d / r^2.
// A step moves bead i by [kappa r_i + D_0 sum_j W_ij F_j] dt plus a random
// displacement of covariance 2 D dt, i.e. sqrt(2 D_0 dt) L xi with L the lower
// Cholesky factor of W and xi the bead normals (RPY is divergence-free, so
// no drift correction).
//
// One CTA integrates one slot (parent or replica) of a chain of N <= 64
// beads, its positions (centre-of-mass frame) in shared memory. The 3N x 3N
// tensor is held as 4 x 4 tiles of its lower triangle in the registers of
// the CTA's threads (tile t of the column-major lower order belongs to
// thread t mod kHIThreads). Per step:
//   - bead forces (springs; Lennard-Jones split over four threads a bead) and
//     bead normals;
//   - the tensor, one 3 x 3 bead block per thread at a time, into a
//     shared-memory copy of the lower tiles, from which each thread loads its
//     own tiles;
//   - the mobility-weighted force u = W F from per-tile partial products,
//     summed in a fixed order (no atomics: the results do not depend on timing);
//   - right-looking blocked Cholesky over tile columns K: the owners of
//     (I, K) solve against the factored (K, K), every owner of a tile (I, J),
//     K < J <= I, subtracts L_IK L_JK^T, and the owner of (K+1, K+1)
//     factors it as soon as its own update is done - two barriers a column;
//   - the correlated noise L xi from per-tile partials, the update and the
//     centre-of-mass shift.
#pragma once

#include "bd_lj.cuh"

namespace bdra {

constexpr int kHIThreads = 256;
constexpr int kHIMaxBeads = 64;
constexpr int kHISmallBeads = 50;
// Tile rows of the largest tensor of each kernel: chains of up to
// kHISmallBeads beads (three tiles per thread, three CTAs per SM in float32) and of up to
// kHIMaxBeads (five tiles per thread).
constexpr int kHINTSmall = (3 * kHISmallBeads + 3) / 4;
constexpr int kHINTMax = (3 * kHIMaxBeads + 3) / 4;

template <int NTM> struct HIDims {
    static constexpr int tiles = NTM * (NTM + 1) / 2;                       // lower tiles
    static constexpr int maxt = (tiles + kHIThreads - 1) / kHIThreads;      // tiles per thread
};

template <typename T, int NTM> struct HIShared {
    static constexpr int kTiles = HIDims<NTM>::tiles;
    static constexpr int kPanel = 20;  // panel row stride: 16-byte rows, conflict-free vector loads
    alignas(16) T pos[4 * NTM];        // bead positions [3N] (COM frame); padding 0
    alignas(16) T frc[4 * NTM];        // bead forces [3N]; padding 0
    alignas(16) T xi[4 * NTM];         // bead normals [3N]; padding 0
    alignas(16) T diag[16];            // factor of the current diagonal tile
    alignas(16) T dinv[4];             // reciprocals of its diagonal
    alignas(16) T panel[NTM][kPanel];  // factor tiles of the current tile column, by tile row
    // bead pairs bi >= bj in row-major order as (bi << 8) | bj, for the chains of this kernel
    static constexpr int kBeads = NTM <= kHINTSmall ? kHISmallBeads : kHIMaxBeads;
    uint16_t pair[kBeads * (kBeads + 1) / 2];
    // W's lower tiles (entry e of tile t at tiles[e][t]) until the threads
    // have loaded theirs, then the per-tile partial products (part[c][t])
    union alignas(16) {
        T tiles[16][kTiles];
        T part[8][kTiles];
    } st;
    T com[3];
};

// Tiles of the lower triangle (I >= J) in column-major order over NT tile
// rows: column J starts at J NT - J (J - 1) / 2. The tiles still to be
// updated at column step K (J > K) are then a suffix of the order, so they
// sit on consecutive threads and finished warps drop out whole.
__device__ __forceinline__ int hi_tile(int I, int J, int NT) { return J * NT - J * (J - 1) / 2 + (I - J); }

__device__ __forceinline__ void hi_uncol(int t, int NT, int& I, int& J)
{
    J = 0;
    while (J + 1 < NT && (J + 1) * NT - (J + 1) * J / 2 <= t) ++J;
    I = J + (t - (J * NT - J * (J - 1) / 2));
}

// Row-major lower-triangle index t = I (I + 1) / 2 + J back to (I, J).
__device__ __forceinline__ void hi_untri(int t, int& I, int& J)
{
    I = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while (I * (I + 1) / 2 > t) --I;
    while ((I + 1) * (I + 2) / 2 <= t) ++I;
    J = t - I * (I + 1) / 2;
}

// The RPY block of two different beads as c_i I + c_d d d^T.
template <typename T, bool FAST>
__device__ __forceinline__ void rpy_coef(T dx, T dy, T dz, T a, T& ci, T& cd)
{
    const T r2 = fma(dx, dx, fma(dy, dy, dz * dz));
    const T ir = Rsqrt<T, FAST>::rsqrt(r2);
    const T r = r2 * ir;
    if (r >= T(2) * a) {
        const T pre = T(0.75) * a * ir;
        const T a2r2 = a * a * ir * ir;
        ci = pre * fma(T(2.0 / 3.0), a2r2, T(1));
        cd = pre * fma(T(-2), a2r2, T(1)) * (ir * ir);
    } else {
        ci = fma(T(-9.0 / 32.0) / a, r, T(1));
        cd = (T(3.0 / 32.0) / a) * ir;
    }
}

// 16 values from / to 16-byte aligned shared memory.
__device__ __forceinline__ void hi_ld16(const float* src, float (&d)[16])
{
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 v = reinterpret_cast<const float4*>(src)[q];
        d[4 * q] = v.x; d[4 * q + 1] = v.y; d[4 * q + 2] = v.z; d[4 * q + 3] = v.w;
    }
}
__device__ __forceinline__ void hi_ld16(const double* src, double (&d)[16])
{
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const double2 v = reinterpret_cast<const double2*>(src)[q];
        d[2 * q] = v.x; d[2 * q + 1] = v.y;
    }
}
__device__ __forceinline__ void hi_st16(float* dst, const float (&d)[16])
{
#pragma unroll
    for (int q = 0; q < 4; ++q)
        reinterpret_cast<float4*>(dst)[q] = make_float4(d[4 * q], d[4 * q + 1], d[4 * q + 2], d[4 * q + 3]);
}
__device__ __forceinline__ void hi_st16(double* dst, const double (&d)[16])
{
#pragma unroll
    for (int q = 0; q < 8; ++q) reinterpret_cast<double2*>(dst)[q] = make_double2(d[2 * q], d[2 * q + 1]);
}

// Per-thread state of the tensor tiles.
template <typename T, int MAXT> struct HITiles {
    T A[MAXT][16];       // row-major 4 x 4
    int I[MAXT], J[MAXT];   // -1: no tile
};

template <typename T, int MAXT>
__device__ __forceinline__ void hi_tiles_init(HITiles<T, MAXT>& tl, int NT)
{
    const int total = NT * (NT + 1) / 2;
#pragma unroll
    for (int s = 0; s < MAXT; ++s) {
        const int t = threadIdx.x + s * kHIThreads;
        int I = -1, J = -1;
        if (t < total) hi_uncol(t, NT, I, J);
        tl.I[s] = I;
        tl.J[s] = J;
    }
}

// The bead pairs of a chain of N beads into sm.pair (once per kernel).
template <typename T, int NTM>
__device__ __forceinline__ void hi_pairs_init(HIShared<T, NTM>& sm, int N)
{
    for (int k = threadIdx.x; k < N * (N + 1) / 2; k += blockDim.x) {
        int bi, bj;
        hi_untri(k, bi, bj);
        sm.pair[k] = (uint16_t)((bi << 8) | bj);
    }
}

// W's lower tiles into sm.st.tiles from the positions: bead pairs bi >= bj,
// spread over the threads; a 3 x 3 block per pair (Eq. 2 on the diagonal,
// Eq. 3 off it). Entries above the diagonal inside a diagonal tile are
// written too (W is symmetric); rows and columns >= 3N are not written.
// Entry (p, q) of tile (I, J) = (p >> 2, q >> 2) is element
// (4 (p & 3) + (q & 3)) kTiles + J NT - J (J + 1) / 2 + I of the tile copy:
// a part of the row p plus a part of the column q.
template <typename T, bool FAST, int NTM>
__device__ __forceinline__ void hi_assemble(HIShared<T, NTM>& sm, int N, T a)
{
    constexpr int kT = HIShared<T, NTM>::kTiles;
    const int pairs = N * (N + 1) / 2;
    const int NT = (3 * N + 3) / 4;
    T* tiles = &sm.st.tiles[0][0];
#pragma unroll 1
    for (int k = threadIdx.x; k < pairs; k += kHIThreads) {
        const int bi = sm.pair[k] >> 8, bj = sm.pair[k] & 0xFF;
        T ci = T(1), cd = T(0), d[3] = {T(0), T(0), T(0)};
        if (bi != bj) {
#pragma unroll
            for (int c = 0; c < 3; ++c) d[c] = sm.pos[3 * bj + c] - sm.pos[3 * bi + c];
            rpy_coef<T, FAST>(d[0], d[1], d[2], a, ci, cd);
        }
        int row[3], rowm[3], I[3], col[3], colm[3], J[3];
#pragma unroll
        for (int x = 0; x < 3; ++x) {
            const int p = 3 * bi + x;
            I[x] = p >> 2;
            row[x] = 4 * (p & 3) * kT + I[x];    // p as the entry's row
            rowm[x] = (p & 3) * kT + I[x];       // p as the mirrored entry's column
        }
#pragma unroll
        for (int y = 0; y < 3; ++y) {
            const int q = 3 * bj + y;
            J[y] = q >> 2;
            const int cs = J[y] * NT - J[y] * (J[y] + 1) / 2;
            col[y] = (q & 3) * kT + cs;
            colm[y] = 4 * (q & 3) * kT + cs;
        }
#pragma unroll
        for (int x = 0; x < 3; ++x)
#pragma unroll
            for (int y = 0; y < 3; ++y) {
                if (bi == bj && x < y) continue;        // diagonal block: lower part (mirrored below)
                T w = cd * d[x] * d[y];
                if (x == y) w += ci;
                tiles[row[x] + col[y]] = w;
                if (I[x] == J[y] && (bi != bj || x != y)) tiles[rowm[x] + colm[y]] = w;
            }
    }
}

// The thread's tiles from sm.st.tiles; rows and columns >= n (the last tile
// row only) are the identity's.
template <typename T, int NTM, int MAXT>
__device__ __forceinline__ void hi_load_tiles(HITiles<T, MAXT>& tl, const HIShared<T, NTM>& sm, int n)
{
#pragma unroll
    for (int s = 0; s < MAXT; ++s) {
        if (tl.I[s] < 0) continue;
        const int I = tl.I[s], J = tl.J[s], t = hi_tile(I, J, (n + 3) >> 2);
#pragma unroll
        for (int e = 0; e < 16; ++e) tl.A[s][e] = sm.st.tiles[e][t];
        if (4 * I + 3 >= n) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int p = 4 * I + i, q = 4 * J + j;
                    if (p >= n || q >= n) tl.A[s][4 * i + j] = p == q ? T(1) : T(0);
                }
        }
    }
}

// Factor of a diagonal tile (lower part; the upper part is left as is) and
// the reciprocals of its diagonal. The fast float form takes both from one
// approximate reciprocal square root.
template <typename T, bool FAST>
__device__ __forceinline__ void hi_chol4(T (&A)[16], T (&inv)[4])
{
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        T s = A[5 * j];
#pragma unroll
        for (int k = 0; k < j; ++k) s = fma(-A[4 * j + k], A[4 * j + k], s);
        T l, il;
        if (FAST) {
            il = Rsqrt<T, FAST>::rsqrt(s);
            l = s * il;
        } else {
            l = sqrt(s);
            il = T(1) / l;
        }
        A[5 * j] = l;
        inv[j] = il;
#pragma unroll
        for (int i = j + 1; i < 4; ++i) {
            T v = A[4 * i + j];
#pragma unroll
            for (int k = 0; k < j; ++k) v = fma(-A[4 * i + k], A[4 * j + k], v);
            A[4 * i + j] = v * il;
        }
    }
}

// X L^T = A for a tile below the diagonal tile L (lower; inv: 1 / its diagonal).
template <typename T>
__device__ __forceinline__ void hi_trsm4(T (&A)[16], const T* L, const T* inv)
{
    T Lr[16], iv[4];
    hi_ld16(L, Lr);
#pragma unroll
    for (int c = 0; c < 4; ++c) iv[c] = inv[c];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            T v = A[4 * r + c];
#pragma unroll
            for (int k = 0; k < c; ++k) v = fma(-A[4 * r + k], Lr[4 * c + k], v);
            A[4 * r + c] = v * iv[c];
        }
}

// In-place lower Cholesky factor of the CTA's tiles (every thread calls it).
// Column step K: the owners of (I, K), I > K, solve against the factored
// diagonal tile; barrier; every owner of a tile (I, J), K < J <= I,
// subtracts L_IK L_JK^T, and the owner of (K+1, K+1), right after its own
// update, factors that tile for the next step (the column-major order makes
// it the thread's first active tile); barrier.
template <typename T, bool FAST, int NTM, int MAXT>
__device__ __forceinline__ void hi_cholesky(HITiles<T, MAXT>& tl, HIShared<T, NTM>& sm, int NT)
{
#pragma unroll
    for (int s = 0; s < MAXT; ++s)
        if (tl.I[s] == 0 && tl.J[s] == 0) {
            T inv[4];
            hi_chol4<T, FAST>(tl.A[s], inv);
            hi_st16(sm.diag, tl.A[s]);
#pragma unroll
            for (int e = 0; e < 4; ++e) sm.dinv[e] = inv[e];
        }
    __syncthreads();
#pragma unroll 1
    for (int K = 0; K < NT; ++K) {
#pragma unroll
        for (int s = 0; s < MAXT; ++s)
            if (tl.J[s] == K && tl.I[s] > K) {
                hi_trsm4(tl.A[s], sm.diag, sm.dinv);
                hi_st16(sm.panel[tl.I[s]], tl.A[s]);
            }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < MAXT; ++s)
            if (tl.J[s] > K) {
                T li[16], lj[16];
                hi_ld16(sm.panel[tl.I[s]], li);
                hi_ld16(sm.panel[tl.J[s]], lj);
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        T v = tl.A[s][4 * i + j];
#pragma unroll
                        for (int k = 0; k < 4; ++k) v = fma(-li[4 * i + k], lj[4 * j + k], v);
                        tl.A[s][4 * i + j] = v;
                    }
                if (tl.I[s] == K + 1 && tl.J[s] == K + 1) {
                    T inv[4];
                    hi_chol4<T, FAST>(tl.A[s], inv);
                    hi_st16(sm.diag, tl.A[s]);
#pragma unroll
                    for (int e = 0; e < 4; ++e) sm.dinv[e] = inv[e];
                }
            }
        __syncthreads();
    }
}

// Bead forces into sm.frc (springs and pair forces): four consecutive
// threads a bead (blockDim.x / 4 beads at a time), the pair sum split over
// them by partner index mod 4 and combined by shuffles in a fixed order.
// Returns the FENE floor count of the thread's springs (the bead's first
// thread).
template <typename T, bool FAST, typename SM>
__device__ __forceinline__ int hi_forces(SM& sm, int N, const StepConst<T, FAST>& k,
                                         const LJConst<T>& kl, bool harmonic, bool lj)
{
    int floored = 0;
    const int q = threadIdx.x & 3;
#pragma unroll 1
    for (int base = 0; base < N; base += (int)(blockDim.x >> 2)) {
    const int b = base + (int)(threadIdx.x >> 2);
    T f[3] = {T(0), T(0), T(0)};
    if (b < N) {
        if (q == 0) {
            // springs b (to bead b+1) and b-1 (from bead b-1)
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const int i = b - side;               // spring index
                if (i < 0 || i + 1 >= N) continue;
                const T qx = sm.pos[3 * i + 3] - sm.pos[3 * i];
                const T qy = sm.pos[3 * i + 4] - sm.pos[3 * i + 1];
                const T qz = sm.pos[3 * i + 5] - sm.pos[3 * i + 2];
                T c;
                if (harmonic) {          // the laws with a rest length (harmonic, vWF)
                    int fl = 0;
                    c = rest_law_coef<T, FAST>(qx, qy, qz, (i & 1) == 0, k.H, kl, k.smin, fl);
                    if (side == 0) floored += fl;
                } else {
                    int fl = 0;
                    c = spring_coef<T, FAST>(qx, qy, qz, k.H, k.Hinvb, k.smin, fl);
                    if (side == 0) floored += fl;
                }
                const T sg = side == 0 ? T(1) : T(-1);
                f[0] = fma(sg * c, qx, f[0]); f[1] = fma(sg * c, qy, f[1]); f[2] = fma(sg * c, qz, f[2]);
            }
        }
        if (lj) {
            const T x0 = sm.pos[3 * b], y0 = sm.pos[3 * b + 1], z0 = sm.pos[3 * b + 2];
#pragma unroll 1
            for (int j = q; j < N; j += 4) {
                if (j == b || j == b - 1 || j == b + 1) continue;
                const T dx = sm.pos[3 * j] - x0, dy = sm.pos[3 * j + 1] - y0, dz = sm.pos[3 * j + 2] - z0;
                const T c = lj_coef<T, FAST>(dx, dy, dz, kl);
                f[0] = fma(c, dx, f[0]); f[1] = fma(c, dy, f[1]); f[2] = fma(c, dz, f[2]);
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        f[c] += __shfl_xor_sync(0xffffffffu, f[c], 1);
        f[c] += __shfl_xor_sync(0xffffffffu, f[c], 2);
    }
    if (b < N && q == 0) {
        sm.frc[3 * b] = f[0];
        sm.frc[3 * b + 1] = f[1];
        sm.frc[3 * b + 2] = f[2];
    }
    }
    return floored;
}

// Positions from bonds [nb][3] (bead 0 at the origin), then the COM shift.
template <typename T, typename SM>
__device__ __forceinline__ void hi_load_bonds(SM& sm, const T* bonds, int N)
{
    __syncthreads();     // every thread is done reading the old positions
    if (threadIdx.x < 3) {
        const int c = threadIdx.x;
        T x = T(0);
        sm.pos[c] = x;
        for (int i = 0; i + 1 < N; ++i) {
            x += bonds[3 * i + c];
            sm.pos[3 * (i + 1) + c] = x;
        }
        T s = T(0);
        for (int i = 0; i < N; ++i) s += sm.pos[3 * i + c];
        sm.com[c] = s / (T)N;
    }
    __syncthreads();
    if (threadIdx.x < 3 * N) sm.pos[threadIdx.x] -= sm.com[threadIdx.x % 3];
    __syncthreads();
}

template <typename T, typename SM>
__device__ __forceinline__ void hi_store_bonds(const SM& sm, T* bonds, int N)
{
    for (int e = threadIdx.x; e < 3 * (N - 1); e += blockDim.x) bonds[e] = sm.pos[e + 3] - sm.pos[e];
}

// One step t -> t + 1 of the CTA's slot. Returns the thread's floor count.
template <typename T, bool FAST, int NTM, int MAXT>
__device__ __forceinline__ int hi_step(HIShared<T, NTM>& sm, HITiles<T, MAXT>& tl, const ChainDev& ch,
                                       const StepConst<T, FAST>& k, const LJConst<T>& kl,
                                       const StepParams& p, int N, int NT,
                                       uint32_t slot_key, uint32_t chain, uint32_t step, bool harmonic,
                                       bool lj)
{
    const int n = 3 * N;
    const int tid = threadIdx.x;
    const int floored = hi_forces<T, FAST>(sm, N, k, kl, harmonic, lj);
    if (tid < N) {
        T z0, z1, z2;
        bead_noise<T, FAST>((uint32_t)tid, slot_key, step, chain, p, z0, z1, z2);
        sm.xi[3 * tid] = z0;
        sm.xi[3 * tid + 1] = z1;
        sm.xi[3 * tid + 2] = z2;
    }
    hi_assemble<T, FAST, NTM>(sm, N, (T)ch.hi_a);
    __syncthreads();
    hi_load_tiles<T, NTM, MAXT>(tl, sm, n);
    __syncthreads();                   // the partial products below overwrite the tile copy
    // u = W F: per tile W_IJ F_J (rows I) and, below the diagonal, W_IJ^T F_I (rows J)
#pragma unroll
    for (int s = 0; s < MAXT; ++s) {
        if (tl.I[s] < 0) continue;
        const int I = tl.I[s], J = tl.J[s], t = hi_tile(I, J, NT);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            T v = T(0);
#pragma unroll
            for (int j = 0; j < 4; ++j) v = fma(tl.A[s][4 * i + j], sm.frc[4 * J + j], v);
            sm.st.part[i][t] = v;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            T v = T(0);
            if (J < I) {
#pragma unroll
                for (int i = 0; i < 4; ++i) v = fma(tl.A[s][4 * i + j], sm.frc[4 * I + i], v);
            }
            sm.st.part[4 + j][t] = v;
        }
    }
    __syncthreads();
    T u = T(0);
    if (tid < n) {
        const int I = tid >> 2, c = tid & 3;
        for (int J = 0; J <= I; ++J) u += sm.st.part[c][hi_tile(I, J, NT)];
        for (int I2 = I + 1; I2 < NT; ++I2) u += sm.st.part[4 + c][hi_tile(I2, I, NT)];
    }
    hi_cholesky<T, FAST, NTM, MAXT>(tl, sm, NT);   // its first barrier also ends the reads of sm.st above
    // w = L xi
#pragma unroll
    for (int s = 0; s < MAXT; ++s) {
        if (tl.I[s] < 0) continue;
        const int I = tl.I[s], J = tl.J[s], t = hi_tile(I, J, NT);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            T v = T(0);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (J < I || j <= i) v = fma(tl.A[s][4 * i + j], sm.xi[4 * J + j], v);
            sm.st.part[i][t] = v;
        }
    }
    __syncthreads();
    T nv = T(0);
    if (tid < n) {
        const int I = tid >> 2, c = tid & 3;
        T w = T(0);
        for (int J = 0; J <= I; ++J) w += sm.st.part[c][hi_tile(I, J, NT)];
        const int x = tid % 3, b3 = tid - x;
        const T r = sm.pos[tid];
        // kappa . r dt: xx, yy, zz and xz (shear) only
        T fl = x == 0 ? fma(k.axz, sm.pos[b3 + 2], fma(k.axx, r, r)) : (x == 1 ? fma(k.ayy, r, r) : fma(k.azz, r, r));
        nv = fma(k.cn, w, fma(k.cd, u, fl));
    }
    __syncthreads();
    if (tid < n) sm.pos[tid] = nv;
    __syncthreads();
    if (tid < 32) {
        T s[3] = {T(0), T(0), T(0)};
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
            for (int c = 0; c < 3; ++c) sm.com[c] = s[c] / (T)N;
    }
    __syncthreads();
    if (tid < n) sm.pos[tid] -= sm.com[tid % 3];
    __syncthreads();
    return floored;
}

// Eq. 5 at a window end (BD_FLAG_CONFORMATION): the replica's COM-frame
// positions against those of the halted parent it was formed from (the
// window-start snapshot, rebuilt from its bonds in sm.frc, which the next
// step overwrites anyway): per bead and component |dr|, their bead means
// (D-bar of this replica) and, for the chain's first replica, R_GZ of the
// parent. The per-bead values go to the replica's own partial row (its
// group), which the window fold averages over the replicas.
template <typename T, typename SM>
__device__ __forceinline__ void hi_conformation(SM& sm, const ItemDev& it, const ChainDev& ch,
                                                const StepParams& p, int64_t w, int kglob)
{
    const int N = ch.N;
    const T* pc = reinterpret_cast<const T*>(p.snap) + ((w % p.win_ring) * p.M + ch.spr_off) * 3;
    if (threadIdx.x < 3) {
        const int c = threadIdx.x;
        T x = T(0), s = T(0);
        sm.frc[c] = x;
        for (int i = 0; i + 1 < N; ++i) {
            x += pc[3 * i + c];
            sm.frc[3 * (i + 1) + c] = x;
            s += x;
        }
        const T cm = s / (T)N;
        T dsum = T(0), z2 = T(0);
        for (int b = 0; b < N; ++b) {
            const T pp = sm.frc[3 * b + c] - cm;
            sm.frc[3 * b + c] = pp;
            dsum += fabs(sm.pos[3 * b + c] - pp);
            z2 = fma(pp, pp, z2);
        }
        p.dbar[((int64_t)w * p.n_rep + ch.rep_off + kglob - 1) * 3 + c] = (double)dsum / N;
        if (c == 2 && it.group == 0) p.rgz[(int64_t)w * p.n_chains + it.chain] = sqrt((double)z2 / N);
    }
    __syncthreads();
    double* out = p.dbead_part + ((w % p.win_ring) * p.bpart_stride + ch.bpart_off + (int64_t)it.group * N) * 3;
    for (int e = threadIdx.x; e < 3 * N; e += blockDim.x) out[e] = (double)fabs(sm.pos[e] - sm.frc[e]);
    __syncthreads();
}

// The CUDA-core engine of a slot: W's lower 4 x 4 tiles in the registers
// of the CTA's threads (hi_step). Engines give the kernel bodies below their
// shared memory, their per-thread state and their step.
template <typename T, bool FAST, int NTM> struct HITileEngine {
    using Shared = HIShared<T, NTM>;
    static constexpr int kMaxT = HIDims<NTM>::maxt;
    HITiles<T, kMaxT> tl;
    int NT;
    __device__ __forceinline__ void begin(Shared& sm, int N, int32_t)
    {
        NT = (3 * N + 3) / 4;
        for (int e = threadIdx.x; e < 4 * NTM; e += blockDim.x) {
            sm.pos[e] = T(0); sm.frc[e] = T(0); sm.xi[e] = T(0);
        }
        hi_pairs_init(sm, N);
        __syncthreads();
        hi_tiles_init(tl, NT);
    }
    __device__ __forceinline__ int step(Shared& sm, const ChainDev& ch, const StepConst<T, FAST>& k,
                                        const LJConst<T>& kl, const StepParams& p, int N, uint32_t key,
                                        uint32_t chain, uint32_t t, bool harmonic, bool lj)
    {
        return hi_step<T, FAST, NTM, kMaxT>(sm, tl, ch, k, kl, p, N, NT, key, chain, t, harmonic, lj);
    }
    __device__ __forceinline__ bool failed() const { return false; }
    __device__ __forceinline__ void end(Shared&, int32_t*) {}
};

// Replicas: one CTA per work item (one replica), the items of this launch in
// p.items. Spawn from the window-start snapshot, S steps, one force sample per
// spring at the window end into the replica's partial row (its group).
template <typename T, bool FAST, typename E>
__device__ __forceinline__ void hi_replica_body(const StepParams& p, typename E::Shared& sm)
{
    if ((int)blockIdx.x >= p.n_items) return;
    const ItemDev it = p.items[blockIdx.x];
    const ChainDev ch = p.chains[it.chain];
    const int N = ch.N, nb = N - 1;
    const bool harmonic = ch.spring == BD_SPRING_HARMONIC || ch.spring == BD_SPRING_VWF;
    LJConst<T> kl;
    kl.load(ch);
    const bool lj = ch.lj_u > 0.0;
    const int kglob = it.rep_begin + 1;
    const uint32_t key = (p.flags & BD_FLAG_IDENTICAL_NOISE) ? 0u : (uint32_t)kglob;
    StepConst<T, FAST> k;
    k.load(ch, p);
    E eng;
    eng.begin(sm, N, p.flags);
    T* state = reinterpret_cast<T*>(p.state) + (ch.state_off + (int64_t)kglob * nb) * 3;
    const T* snap = reinterpret_cast<const T*>(p.snap);
    hi_load_bonds(sm, state, N);
    int floored = 0;
    int s_in = (int)(p.t0 % p.S);
    int64_t w = p.t0 / p.S;
    const int64_t t_end = p.t0 + p.n_steps;
#pragma unroll 1
    for (int64_t t = p.t0; t < t_end; ++t) {
        if (s_in == 0) hi_load_bonds(sm, snap + ((w % p.win_ring) * p.M + ch.spr_off) * 3, N);
        floored += eng.step(sm, ch, k, kl, p, N, key, (uint32_t)it.chain + p.chain_base, (uint32_t)t, harmonic, lj);
        if (eng.failed()) break;
        if (++s_in == p.S) {
            s_in = 0;
            const int i = threadIdx.x;
            if (i < nb) {
                const T qx = sm.pos[3 * i + 3] - sm.pos[3 * i];
                const T qy = sm.pos[3 * i + 4] - sm.pos[3 * i + 1];
                const T qz = sm.pos[3 * i + 5] - sm.pos[3 * i + 2];
                const T f = harmonic ? rest_law_tension<T, FAST>(qx, qy, qz, (i & 1) == 0, k.H, kl, k.smin)
                                     : spring_tension<T, FAST>(qx, qy, qz, k.H, k.Hinvb, k.smin);
                p.part_hist[(w % p.win_ring) * p.part_stride + ch.part_off + (int64_t)it.group * nb + i] = (double)f;
            }
            if (p.flags & BD_FLAG_CONFORMATION) hi_conformation<T>(sm, it, ch, p, w, kglob);
            ++w;
        }
    }
    eng.end(sm, p.dev_err);
    hi_store_bonds(sm, state, N);
    if (floored) atomicAdd(p.overext + it.chain, (unsigned long long)floored);
}

// Parents: one CTA per chain (p.parent_warps[blockIdx.x].first indexes
// p.parent_items). Window-start snapshots, then per step the update and the
// instantaneous force of every spring: TSF sums and the ISF criteria.
template <typename T, bool FAST, typename E>
__device__ __forceinline__ void hi_parent_body(const StepParams& p, typename E::Shared& sm)
{
    if ((int)blockIdx.x >= p.n_parent_warps) return;
    const int c = p.parent_items[p.parent_warps[blockIdx.x].first];
    const ChainDev ch = p.chains[c];
    const int N = ch.N, nb = N - 1;
    const bool harmonic = ch.spring == BD_SPRING_HARMONIC || ch.spring == BD_SPRING_VWF;
    LJConst<T> kl;
    kl.load(ch);
    const bool lj = ch.lj_u > 0.0;
    StepConst<T, FAST> k;
    k.load(ch, p);
    E eng;
    eng.begin(sm, N, p.flags);
    T* state = reinterpret_cast<T*>(p.state) + ch.state_off * 3;
    T* snap = reinterpret_cast<T*>(p.snap);
    hi_load_bonds(sm, state, N);
    const int64_t M = p.M;
    const int i = threadIdx.x;                 // this thread's spring
    const bool mine = i < nb;
    const int64_t m = ch.spr_off + i;
    const bool isf_thr = (p.thr_mask & BD_CRIT_ISF) != 0;
    const bool isf_bell = (p.bell_mask & BD_CRIT_ISF) != 0;
    const T fc = (T)ch.f_c;
    BellConst bk;
    bk.load(ch.k0, p.dt, ch.dx);
    ParentSums<T> sums;     // time-average sum and window hazard: float64, or float-float pairs
    sums.start(mine ? p.tsf_acc[m] : 0.0, mine ? p.exp1[CRIT_Q_ISF * M + m] - p.lam[CRIT_Q_ISF * M + m] : 0.0);
    const bool quiet = ch.spring == BD_SPRING_VWF && (i & 1);   // disulfide bonds do not unfold
    bool thr_done = !mine || quiet || p.first_thr[CRIT_Q_ISF * M + m] >= 0;
    bool bell_done = !mine || quiet || p.first_bell[CRIT_Q_ISF * M + m] >= 0;
    int floored = 0;
    int s_in = (int)(p.t0 % p.S);
    int64_t w = p.t0 / p.S;
    const int64_t t_end = p.t0 + p.n_steps;
#pragma unroll 1
    for (int64_t t = p.t0; t < t_end; ++t) {
        if (s_in == 0) {  // the conformation the replicas of window w start from
            T* row = snap + ((w % p.win_ring) * M + ch.spr_off) * 3;
            hi_store_bonds(sm, row, N);
            // continue from it as the replicas do, so that replicas drawing
            // the parent's noise repeat the parent exactly
            hi_load_bonds(sm, row, N);
        }
        floored += eng.step(sm, ch, k, kl, p, N, 0u, (uint32_t)c + p.chain_base, (uint32_t)t, harmonic, lj);
        if (eng.failed()) break;
        if (mine) {
            const T qx = sm.pos[3 * i + 3] - sm.pos[3 * i];
            const T qy = sm.pos[3 * i + 4] - sm.pos[3 * i + 1];
            const T qz = sm.pos[3 * i + 5] - sm.pos[3 * i + 2];
            const T f = harmonic ? rest_law_tension<T, FAST>(qx, qy, qz, (i & 1) == 0, k.H, kl, k.smin)
                                 : spring_tension<T, FAST>(qx, qy, qz, k.H, k.Hinvb, k.smin);
            sums.add_isf(f);
            if (isf_thr && !thr_done && f >= fc) {
                thr_done = true;
                p.first_thr[CRIT_Q_ISF * M + m] = t + 1;
            }
            if (isf_bell && !quiet) {
                const bool reached = sums.add_hazard(f, bk, p.lam + CRIT_Q_ISF * M + m);
                if (!bell_done && reached) {
                    bell_done = true;
                    p.first_bell[CRIT_Q_ISF * M + m] = t + 1;
                }
            }
        }
        if (++s_in == p.S) {
            s_in = 0;
            if (mine) {
                p.tsf_hist[w * M + m] = sums.tsf_sum() / (double)p.S;
                double rem = 0.0;
                if (isf_bell) {
                    const double lam = p.lam[CRIT_Q_ISF * M + m] + sums.hazard();
                    p.lam[CRIT_Q_ISF * M + m] = lam;
                    rem = p.exp1[CRIT_Q_ISF * M + m] - lam;
                }
                sums.next_window(rem);
            }
            ++w;
        }
    }
    eng.end(sm, p.dev_err);
    __syncthreads();
    hi_store_bonds(sm, state, N);
    if (mine) {
        p.tsf_acc[m] = sums.tsf_sum();
        if (isf_bell) p.lam[CRIT_Q_ISF * M + m] += sums.hazard();
    }
    if (floored) atomicAdd(p.overext + c, (unsigned long long)floored);
}

template <typename T, bool FAST, int NTM>
__global__ void __launch_bounds__(kHIThreads, (sizeof(T) == 4 && NTM <= kHINTSmall) ? 3 : 1)
hi_replica_kernel(const StepParams p)
{
    extern __shared__ __align__(16) unsigned char hi_smem_raw[];
    hi_replica_body<T, FAST, HITileEngine<T, FAST, NTM>>(p, *reinterpret_cast<HIShared<T, NTM>*>(hi_smem_raw));
}

template <typename T, bool FAST, int NTM>
__global__ void __launch_bounds__(kHIThreads, (sizeof(T) == 4 && NTM <= kHINTSmall) ? 3 : 1)
hi_parent_kernel(const StepParams p)
{
    extern __shared__ __align__(16) unsigned char hi_smem_raw[];
    hi_parent_body<T, FAST, HITileEngine<T, FAST, NTM>>(p, *reinterpret_cast<HIShared<T, NTM>*>(hi_smem_raw));
}

}  // namespace bdra
