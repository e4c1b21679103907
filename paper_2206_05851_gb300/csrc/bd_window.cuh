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
#include "bd_lj.cuh"
#include "bd_step.cuh"

namespace bdra {

// ---------------------------------------------------------------------------
// Replicas, one warp work item (one replica per lane run). Lane run s of the
// warp is replica rep_begin + stride s + 1; state of replica k lives at
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
// the step loop carries no trace of them. H: the noise half of every replica
// of the item (known when all are odd or all even), or -1.
template <typename T, int L, bool FAST, bool TAB, bool CONF, bool LJ, int H>
__device__ __forceinline__ void run_one_item_h(const ItemDev& it, const StepParams& p, T* wsm,
                                               uint4* ptab)
{
    const ChainDev ch = p.chains[it.chain];
    const int nb = ch.N - 1;
    const int G = (ch.N + L - 1) / L;
    const int P = 32 / G;
    const int lane = threadIdx.x & 31;
    const int sw = lane / G;
    const bool active = (sw < P) && (sw < it.rep_count);
    const int kglob = it.rep_begin + it.stride * sw + 1;
    const uint32_t key = (p.flags & BD_FLAG_IDENTICAL_NOISE) ? 0u : (uint32_t)kglob;
    const LaneCtx lc = make_lane(sw < P ? lane - sw * G : 0, G, L, lane, nb, active, key,
                                 (uint32_t)it.chain + p.chain_base);
    StepConst<T, FAST> k;
    k.load(ch, p);
    LJConst<T> kl;
    if (LJ) kl.load(ch);
    if (TAB) {
        for (int b = lane; b < G * L; b += 32)
            ptab[b] = PhiloxSplit::bead_part((uint32_t)b, (uint32_t)it.chain + p.chain_base, p.rk0, p.rk1);
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
        if constexpr (LJ)
            floored += step_bonds_lj<T, L, FAST, TAB, H>(qx, qy, qz, lc, k, kl, sw < P, sw < P ? lane - sw * G : 0, G,
                                           sw < P ? sw * G : lane, (uint32_t)t, p, ptab);
        else
            floored += step_bonds<T, L, FAST, TAB, H>(qx, qy, qz, lc, k, (uint32_t)t, p, ptab);
        if (++s_in == p.S) {
            // one force sample per replica at the end of the evolution time
            s_in = 0;
            if (active) {
#pragma unroll
                for (int j = 0; j < L; ++j) {
                    const int i = lc.bead0 + j;
                    if (i < nb)
                        wsm[sw * nb + i] =
                            LJ ? rest_law_tension<T, FAST>(qx[j], qy[j], qz[j], (i & 1) == 0, k.H, kl, k.smin)
                               : spring_tension<T, FAST>(qx[j], qy[j], qz[j], k.H, k.Hinvb, k.smin);
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

// A work item with one replica per lane run. The planner gives such an item
// only odd or only even replicas (stride 2) or a single one, so all its
// replicas draw the same half of their noise pairs' generator outputs (in
// identical-noise runs all draw the parent's, half 0): the half is fixed
// for the whole warp and compiled in.
template <typename T, int L, bool FAST, bool TAB = false, bool CONF = false, bool LJ = false>
__device__ __forceinline__ void run_one_item(const ItemDev& it, const StepParams& p, T* wsm,
                                             uint4* ptab = nullptr)
{
    const bool h1 = (p.flags & BD_FLAG_IDENTICAL_NOISE) == 0 && noise_half((uint32_t)it.rep_begin + 1u) == 1u;
    if (h1) run_one_item_h<T, L, FAST, TAB, CONF, LJ, 1>(it, p, wsm, ptab);
    else run_one_item_h<T, L, FAST, TAB, CONF, LJ, 0>(it, p, wsm, ptab);
}

// ---------------------------------------------------------------------------
// Parents. Global warp g holds parent_warps[g].count parents (chains
// parent_items[first + s]), each on G lanes.
// Per step: update, then sample the parent's spring forces (ISF): TSF window
// sums and ISF threshold / Bell criteria. Window sums and the window's hazard
// stay in registers; the integrated hazard lives in p.lam (float64).
// ---------------------------------------------------------------------------
template <typename T, int L, bool FAST, bool LJ = false>
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
                                 (uint32_t)c + p.chain_base);
    StepConst<T, FAST> k;
    k.load(ch, p);
    LJConst<T> kl;
    if (LJ) kl.load(ch);
    uint4* ptab = ptab_all[threadIdx.x >> 5];
    for (int e = lane; e < P * G * L; e += 32) {
        const int s2 = e / (G * L);
        const int c2 = p.parent_items[pw.first + min(s2, pw.count - 1)];
        ptab[e] = PhiloxSplit::bead_part((uint32_t)(e - s2 * G * L), (uint32_t)c2 + p.chain_base, p.rk0, p.rk1);
    }
    __syncwarp();
    const uint4* my_tab = ptab + (sw < P ? sw : 0) * G * L;
    const int64_t M = p.M;
    const bool isf_thr = (p.thr_mask & BD_CRIT_ISF) != 0;
    const bool isf_bell = (p.bell_mask & BD_CRIT_ISF) != 0;
    const T fc = (T)ch.f_c;
    BellConst bk;
    bk.load(ch.k0, p.dt, ch.dx);

    T* state = reinterpret_cast<T*>(p.state) + ch.state_off * 3;
    T* snap = reinterpret_cast<T*>(p.snap);
    T qx[L], qy[L], qz[L];
    load_bonds<T, L>(qx, qy, qz, state, lc);

    // per-spring sampling state of this lane's springs: the time-average sum
    // and the Bell hazard in float64, or float-float pairs with float32
    // integration (a plain float32 sum over a 1500-step window would lose
    // about three digits of the TSF before the division)
    ParentSums<T> sums[L];
    // quiet: springs outside the criteria (the disulfide bonds of a vWF chain)
    uint32_t thr_done = 0, bell_done = 0, quiet = 0;
#pragma unroll
    for (int j = 0; j < L; ++j) {
        const int i = lc.bead0 + j;
        const int64_t m = ch.spr_off + i;
        const bool v = active && i < nb;
        sums[j].start(v ? p.tsf_acc[m] : 0.0, v ? p.exp1[CRIT_Q_ISF * M + m] - p.lam[CRIT_Q_ISF * M + m] : 0.0);
        if (ch.spring == BD_SPRING_VWF && (i & 1)) quiet |= 1u << j;
        if (!v || p.first_thr[CRIT_Q_ISF * M + m] >= 0) thr_done |= 1u << j;
        if (!v || p.first_bell[CRIT_Q_ISF * M + m] >= 0) bell_done |= 1u << j;
    }
    thr_done |= quiet;
    bell_done |= quiet;

    int floored = 0;
    int s_in = (int)(p.t0 % p.S);
    int64_t w = p.t0 / p.S;
    const int64_t t_end = p.t0 + p.n_steps;
#pragma unroll 1
    for (int64_t t = p.t0; t < t_end; ++t) {
        if (s_in == 0)   // the conformation the replicas of window w start from
            store_bonds<T, L>(qx, qy, qz, snap + ((w % p.win_ring) * M + ch.spr_off) * 3, lc);
        if constexpr (LJ)
            floored += step_bonds_lj<T, L, FAST, true, 0>(qx, qy, qz, lc, k, kl, sw < P, sw < P ? lane - sw * G : 0, G,
                                            sw < P ? sw * G : lane, (uint32_t)t, p, my_tab);
        else
            floored += step_bonds<T, L, FAST, true, 0>(qx, qy, qz, lc, k, (uint32_t)t, p, my_tab);
        if (active) {
#pragma unroll
            for (int j = 0; j < L; ++j) {
                const int i = lc.bead0 + j;
                if (i < nb) {
                    const T f = LJ ? rest_law_tension<T, FAST>(qx[j], qy[j], qz[j], (i & 1) == 0, k.H, kl, k.smin)
                                   : spring_tension<T, FAST>(qx[j], qy[j], qz[j], k.H, k.Hinvb, k.smin);
                    sums[j].add_isf(f);
                    if (isf_thr && !(thr_done & (1u << j)) && f >= fc) {
                        thr_done |= 1u << j;
                        p.first_thr[CRIT_Q_ISF * M + ch.spr_off + i] = t + 1;
                    }
                    if (isf_bell && !(quiet & (1u << j))) {
                        const bool reached = sums[j].add_hazard(f, bk, p.lam + CRIT_Q_ISF * M + ch.spr_off + i);
                        if (!(bell_done & (1u << j)) && reached) {
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
                        p.tsf_hist[w * M + m] = sums[j].tsf_sum() / (double)p.S;
                        double rem = 0.0;
                        if (isf_bell) {
                            const double lam = p.lam[CRIT_Q_ISF * M + m] + sums[j].hazard();
                            p.lam[CRIT_Q_ISF * M + m] = lam;
                            rem = p.exp1[CRIT_Q_ISF * M + m] - lam;
                        }
                        sums[j].next_window(rem);
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
                p.tsf_acc[m] = sums[j].tsf_sum();
                if (isf_bell) p.lam[CRIT_Q_ISF * M + m] += sums[j].hazard();
            }
        }
    }
    if (floored) atomicAdd(p.overext + c, (unsigned long long)floored);
}

}  // namespace bdra
