// Conformation diagnostics of Eq. 5 (Sec. III) at a window end, computed by
// the replica kernels from the bonds: between a replica after the evolution
// time and the halted parent it was formed from (the window-start snapshot),
// the COM-frame position difference of bead b is
//   D(b) = |dr_b - dcm|,  dr_b = sum_{m<b} (Q_m - P_m),  dcm = (1/N) sum_b dr_b
// (bead 0's offset cancels between the two COM frames), D-bar is its bead
// mean per component, and R_GZ of the parent is the rms of its COM-frame z.
// A slot is a run of G lanes holding L bonds each (lane seg has bonds from
// bead0 = seg L, as in the step kernels); prefix
// sums and totals over a slot are warp-shuffle scans restricted to the run.
// These functions are called by every lane of the warp, at window ends only,
// and are kept out of line so that they add nothing to the step's registers.
// Arithmetic is in the integration precision: the positions summed are of
// bond differences (order one), so float keeps the differences to about
// 1e-6 relative while the float64 pipe, slow on this GPU, stays idle.
#pragma once

#include "bd_device.cuh"

namespace bdra {

struct SlotRun {
    int seg;    // lane's position in its slot (0 for lanes outside any slot)
    int G;      // lanes per slot
    int last;   // lane holding the slot's last segment (the lane itself outside slots)
};

__device__ __forceinline__ SlotRun slot_run(int lane, int sw, int P, int G)
{
    SlotRun r;
    const bool in = sw < P;
    r.seg = in ? lane - sw * G : 0;
    r.G = G;
    r.last = in ? sw * G + G - 1 : lane;
    return r;
}

// Inclusive prefix sum over the lanes of each slot (lanes outside slots get
// junk they never use).
template <typename T>
__device__ __forceinline__ T slot_scan(T v, const SlotRun& r)
{
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const T u = __shfl_up_sync(0xffffffffu, v, d);
        if (r.seg >= d) v += u;
    }
    return v;
}

// Total over the lanes of each slot, on every lane of the slot.
template <typename T>
__device__ __forceinline__ T slot_total(T v, const SlotRun& r)
{
    return __shfl_sync(0xffffffffu, slot_scan(v, r), r.last);
}

// One replica: adds D(b) of the lane's beads to acc and, if dbar3 is not
// NULL, the slot's last lane writes D-bar (3 components). q: the replica's
// bonds [nb][3], pc: the parent's window-start bonds [nb][3]. act: this lane
// holds the replica.
template <typename T, int L>
__device__ __noinline__ void eq5_replica(const T* q, const T* pc, int bead0,
                                         const SlotRun& r, int N, bool act, T (&acc)[L][3],
                                         double* dbar3)
{
    const int nb = N - 1;
    T dq[L][3], s[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int j = 0; j < L; ++j) {
        const int b = bead0 + j;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            dq[j][c] = (act && b < nb) ? q[3 * b + c] - pc[3 * b + c] : T(0);
            s[c] += dq[j][c];
        }
    }
    T pos[L][3], psum[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        T x = slot_scan(s[c], r) - s[c];          // position of the lane's first bead
#pragma unroll
        for (int j = 0; j < L; ++j) {
            pos[j][c] = x;
            if (bead0 + j < N) psum[c] += x;
            x += dq[j][c];
        }
    }
    T dsum[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const T cm = slot_total(psum[c], r) / (T)N;
        T ds = T(0);
#pragma unroll
        for (int j = 0; j < L; ++j) {
            if (bead0 + j < N) {
                const T d = fabs(pos[j][c] - cm);
                ds += d;
                if (act) acc[j][c] += d;
            }
        }
        dsum[c] = slot_total(ds, r);
    }
    if (act && dbar3 && threadIdx.x % 32 == r.last)
        for (int c = 0; c < 3; ++c) dbar3[c] = (double)dsum[c] / N;
}

// R_GZ of the parent conformation pc (bonds [nb][3]); the slot's last lane
// writes it to *out when `write`.
template <typename T, int L>
__device__ __noinline__ void eq5_rgz(const T* pc, int bead0, const SlotRun& r, int N,
                                     bool write, double* out)
{
    const int nb = N - 1;
    T dz[L], s = T(0);
#pragma unroll
    for (int j = 0; j < L; ++j) {
        const int b = bead0 + j;
        dz[j] = b < nb ? pc[3 * b + 2] : T(0);
        s += dz[j];
    }
    T z = slot_scan(s, r) - s, zs = T(0);
    T zb[L];
#pragma unroll
    for (int j = 0; j < L; ++j) {
        zb[j] = z;
        if (bead0 + j < N) zs += z;
        z += dz[j];
    }
    const T zc = slot_total(zs, r) / (T)N;
    T v = T(0);
#pragma unroll
    for (int j = 0; j < L; ++j)
        if (bead0 + j < N) v += (zb[j] - zc) * (zb[j] - zc);
    v = slot_total(v, r);
    if (write && threadIdx.x % 32 == r.last) *out = sqrt((double)v / N);
}

// Sum of acc over the first n_slots slots of the warp (same bead, every
// slot), written by the lanes of slot 0 to out[N][3] (this work item's
// per-bead partial row). Runs on every lane.
template <typename T, int L>
__device__ __noinline__ void eq5_beads_out(const T (&acc)[L][3], int bead0,
                                           const SlotRun& r, int sw, int P, int N, int n_slots,
                                           double* out)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < L; ++j)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            T v = T(0);
            for (int s2 = 0; s2 < P; ++s2) {
                const T u = __shfl_sync(0xffffffffu, acc[j][c], sw < P ? s2 * r.G + r.seg : lane);
                if (s2 < n_slots) v += u;
            }
            if (sw == 0 && bead0 + j < N) out[3 * (bead0 + j) + c] = (double)v;
        }
}

}  // namespace bdra
