// Reverse-mode (adjoint) derivatives of the replica-averaged spring force
// (RSF, Sec. II) and of the Bell log-survival on it (Sec. III) with respect
// to each chain's strain rate, FENE extensibility b and spring constant H:
// pathwise derivatives of the discrete Eq. 1 map with the noise frozen. The
// noise term of Eq. 1 depends neither on the state nor on the parameters, so
// it drops out of the adjoint recursion; it only enters through the
// recomputed trajectory, which is bitwise the forward one.
//
// For one step Q' = Q + dt kappa Q + (dt/4)(F_{i+1} - 2 F_i + F_{i-1}) + noise,
// with F = c(|Q|^2) Q, c = H / s, s = max(1 - (H/b)|Q|^2, s_min):
//   lambda_j  = lambda'_j + dt kappa^T lambda'_j + (dt/4) J_j Lambda_j,
//   Lambda_j  = lambda'_{j-1} - 2 lambda'_j + lambda'_{j+1}  (0 past the ends),
//   J_j v     = c v + 2 (dc/d|Q|^2) (Q.v) Q           (symmetric),
//   dL/drate += dt lambda'_j . (khat Q_j),  kappa = rate khat,
//   dL/dH    += (dt/4) (dc/dH) Q_j . Lambda_j,
//   dL/db    += (dt/4) (dc/db) Q_j . Lambda_j.
// On the FENE floor c = H / s_min: dc/dH = 1/s_min, no other slope.
// The RSF of window w is (1/R) sum_k f(Q^k), f = c |Q|, sampled at the window
// end; its gradient seeds each replica's adjoint there. Replicas copy the
// parent at the window start, so the sum over a window's replicas of their
// adjoints at the start (mu_w) is added to the parent's adjoint when the
// parent's backward sweep passes that step.
//
// Storage: parent conformations every K steps (checkpoints kept by the
// forward pass), a recomputed K-step segment of parent states, and the
// recomputed states of a batch of replica windows.
#pragma once

#include "bd_window.cuh"

namespace bdra {

// Reciprocal for the derivative factors: the hardware approximation in float
// (about one ulp), a correctly rounded division in double.
template <typename T> __device__ __forceinline__ T adj_recip(T x) { return T(1) / x; }
template <> __device__ __forceinline__ float adj_recip<float>(float x) { return rcp_approx(x); }

// Spring-law factors at Q: c = H/s and its slopes (on the floor only dc/dH).
template <typename T>
struct SpringD {
    T c, dcq, dcH, dcb;
    __device__ __forceinline__ void at(T q2, T H, T Hinvb, T smin)
    {
        const T s = fma(-Hinvb, q2, T(1));
        if (s < smin) {
            const T is = adj_recip(smin);
            c = H * is; dcq = T(0); dcH = is; dcb = T(0);
        } else {
            const T is = adj_recip(s);
            const T is2 = is * is;
            c = H * is;
            dcq = H * Hinvb * is2;              // H^2 / (b s^2)
            dcH = is2;                          // 1 / s^2
            dcb = -(Hinvb * Hinvb) * q2 * is2;  // -H^2 |Q|^2 / (b^2 s^2)
        }
    }
};

// kappa dt and khat dt of a chain.
template <typename T>
struct AdjFlow {
    T kxx, kyy, kzz, kxz;
    T hxx, hyy, hzz, hxz;
    __device__ __forceinline__ void load(const ChainDev& ch, const AdjChain& a, double dt)
    {
        kxx = (T)(ch.kxx * dt); kyy = (T)(ch.kyy * dt); kzz = (T)(ch.kzz * dt); kxz = (T)(ch.kxz * dt);
        hxx = (T)(a.khat[0] * dt); hyy = (T)(a.khat[1] * dt); hzz = (T)(a.khat[2] * dt);
        hxz = (T)(a.khat[3] * dt);
    }
};

template <typename T>
struct AdjConst {
    T H, Hinvb, smin, cd;
    AdjFlow<T> fl;
    __device__ __forceinline__ void load(const ChainDev& ch, const AdjChain& a, const StepParams& p)
    {
        H = (T)ch.H; Hinvb = (T)ch.Hinvb; smin = (T)p.s_min; cd = (T)(0.25 * p.dt);
        fl.load(ch, a, p.dt);
    }
};

// Parameter gradients of one lane: partials in the integration precision
// over blocks of 16 steps, folded into float64.
template <typename T>
struct GradAcc {
    T part[3];
    double sum[3];
    int n;
    __device__ __forceinline__ void init()
    {
        part[0] = part[1] = part[2] = T(0);
        sum[0] = sum[1] = sum[2] = 0.0;
        n = 0;
    }
    __device__ __forceinline__ void fold()
    {
#pragma unroll
        for (int j = 0; j < 3; ++j) { sum[j] += (double)part[j]; part[j] = T(0); }
        n = 0;
    }
    __device__ __forceinline__ void tick()
    {
        if (++n == 16) fold();
    }
};

// The lane's L bonds of a stored state (slot row [N-1][3]); zero past the
// lane's springs.
template <typename T, int L>
__device__ __forceinline__ void load_lane(const T* q, const LaneCtx& lc, T (&x)[L], T (&y)[L],
                                          T (&z)[L])
{
#pragma unroll
    for (int j = 0; j < L; ++j) {
        if (j < lc.nv) {
            const int i = lc.bead0 + j;
            x[j] = q[3 * i + 0]; y[j] = q[3 * i + 1]; z[j] = q[3 * i + 2];
        } else {
            x[j] = T(0); y[j] = T(0); z[j] = T(0);
        }
    }
}

// One adjoint step of the lane's L bonds: lx/ly/lz hold lambda at t+1 on
// entry and lambda at t on exit; qx/qy/qz hold the state at t. Adds the
// step's parameter gradients to g. Every lane of the warp calls it.
template <typename T, int L>
__device__ __forceinline__ void adjoint_step(const T (&qx)[L], const T (&qy)[L], const T (&qz)[L],
                                             T (&lx)[L], T (&ly)[L], T (&lz)[L],
                                             const LaneCtx& lc, const AdjConst<T>& k, T (&g)[3])
{
    T pmx = shfl(lx[L - 1], lc.src_prev), pmy = shfl(ly[L - 1], lc.src_prev), pmz = shfl(lz[L - 1], lc.src_prev);
    T pnx = shfl(lx[0], lc.src_next), pny = shfl(ly[0], lc.src_next), pnz = shfl(lz[0], lc.src_next);
    if (!lc.has_prev) { pmx = T(0); pmy = T(0); pmz = T(0); }
    if (!lc.has_next) { pnx = T(0); pny = T(0); pnz = T(0); }
    T mx = pmx, my = pmy, mz = pmz;          // lambda'_{j-1}
#pragma unroll
    for (int j = 0; j < L; ++j) {
        const T cx = lx[j], cy = ly[j], cz = lz[j];
        T nx, ny, nz;
        if (j + 1 < L) { nx = lx[j + 1]; ny = ly[j + 1]; nz = lz[j + 1]; }
        else { nx = pnx; ny = pny; nz = pnz; }
        if (j < lc.nv) {
            const T qxj = qx[j], qyj = qy[j], qzj = qz[j];
            const T Lx = fma(T(-2), cx, mx + nx), Ly = fma(T(-2), cy, my + ny), Lz = fma(T(-2), cz, mz + nz);
            SpringD<T> sd;
            sd.at(fma(qxj, qxj, fma(qyj, qyj, qzj * qzj)), k.H, k.Hinvb, k.smin);
            const T qL = fma(qxj, Lx, fma(qyj, Ly, qzj * Lz));
            const T a = T(2) * sd.dcq * qL;
            lx[j] = fma(k.cd, fma(sd.c, Lx, a * qxj), fma(k.fl.kxx, cx, cx));
            ly[j] = fma(k.cd, fma(sd.c, Ly, a * qyj), fma(k.fl.kyy, cy, cy));
            lz[j] = fma(k.cd, fma(sd.c, Lz, a * qzj), fma(k.fl.kzz, cz, fma(k.fl.kxz, cx, cz)));
            g[0] = fma(cx, fma(k.fl.hxx, qxj, k.fl.hxz * qzj), fma(cy, k.fl.hyy * qyj, fma(cz, k.fl.hzz * qzj, g[0])));
            g[1] = fma(k.cd * sd.dcb, qL, g[1]);
            g[2] = fma(k.cd * sd.dcH, qL, g[2]);
        }
        mx = cx; my = cy; mz = cz;
    }
}

// Lane context of a parent warp (the packing of parent_kernel).
struct ParentLane {
    LaneCtx lc;
    int chain;
};

template <int L>
__device__ __forceinline__ bool parent_lane(const StepParams& p, ParentLane& out)
{
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (gw >= p.n_parent_warps) return false;          // whole warp
    const ParentWarp pw = p.parent_warps[gw];
    const int G = pw.G, P = 32 / G, sw = lane / G;
    const bool active = (sw < P) && (sw < pw.count);
    out.chain = p.parent_items[pw.first + (active ? sw : 0)];
    const int nb = p.chains[out.chain].N - 1;
    out.lc = make_lane(sw < P ? lane - sw * G : 0, G, L, lane, nb, active, 0u,
                       (uint32_t)out.chain + p.chain_base);
    return true;
}

// Fills a parent warp's split-Philox table (parent s at [s G L, (s + 1) G L))
// and returns this lane's part of it.
template <int L>
__device__ __forceinline__ const uint4* parent_table(const StepParams& p, uint4* tab)
{
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const ParentWarp pw = p.parent_warps[gw];
    const int G = pw.G, P = 32 / G, sw = lane / G;
    for (int e = lane; e < P * G * L; e += 32) {
        const int s2 = e / (G * L);
        const int c2 = p.parent_items[pw.first + min(s2, pw.count - 1)];
        tab[e] = PhiloxSplit::bead_part((uint32_t)(e - s2 * G * L), (uint32_t)c2 + p.chain_base, p.rk0, p.rk1);
    }
    __syncwarp();
    return tab + (sw < P ? sw : 0) * G * L;
}

// ---------------------------------------------------------------------------
// Parent recompute: checkpoint ckpt_index (the parent at seg_t0 = t0) ->
// segbuf rows 0 .. n_steps (the states at steps t0 .. t0 + n_steps).
// ---------------------------------------------------------------------------
template <typename T, int L, bool FAST>
__global__ void __launch_bounds__(kAdjThreads) adj_parent_recompute_kernel(const AdjParams a)
{
    __shared__ uint4 tab_all[kAdjThreads / 32][32 * L];    // split-Philox bead parts per warp
    const StepParams& p = a.sp;
    ParentLane pl;
    if ((int)(threadIdx.x >> 5) >= kAdjThreads / 32) return;
    if (!parent_lane<L>(p, pl)) return;
    const ChainDev ch = p.chains[pl.chain];
    StepConst<T, FAST> k;
    k.load(ch, p);
    const uint4* tab = parent_table<L>(p, tab_all[threadIdx.x >> 5]);
    const T* ck = reinterpret_cast<const T*>(a.ckpt) + (a.ckpt_index * p.M + ch.spr_off) * 3;
    T* seg = reinterpret_cast<T*>(a.segbuf) + ch.spr_off * 3;
    T qx[L], qy[L], qz[L];
    load_bonds<T, L>(qx, qy, qz, ck, pl.lc);
    store_bonds<T, L>(qx, qy, qz, seg, pl.lc);
#pragma unroll 1
    for (int s = 0; s < a.n_steps; ++s) {
        step_bonds<T, L, FAST, true>(qx, qy, qz, pl.lc, k, (uint32_t)(a.t0 + s), p, tab);
        store_bonds<T, L>(qx, qy, qz, seg + (int64_t)(s + 1) * p.M * 3, pl.lc);
    }
}

// ---------------------------------------------------------------------------
// Replica windows w = w_batch0 + blockIdx.y (one warp = one work item):
// recompute the S steps from the parent state at the window start (segbuf),
// keeping every state; seed lambda = (G_w / R) grad f at the window end; S
// adjoint steps back; then mu_w of the item's replicas. Each lane reads back
// only the bonds it wrote itself, so the two sweeps need no synchronisation.
// ---------------------------------------------------------------------------
template <typename T, int L, bool FAST>
__global__ void __launch_bounds__(kAdjThreads) adj_replica_window_kernel(const AdjParams a)
{
    __shared__ uint4 tab_all[kAdjThreads / 32][32 * L];    // split-Philox bead parts per warp
    const StepParams& p = a.sp;
    if ((int)(threadIdx.x >> 5) >= kAdjThreads / 32) return;
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (gw >= a.n_items) return;                        // whole warp
    const ItemDev it = a.items[gw];
    const ChainDev ch = p.chains[it.chain];
    const AdjChain ac = a.adj[it.chain];
    const int nb = ch.N - 1;
    const int G = (ch.N + L - 1) / L, P = 32 / G;
    const int lane = threadIdx.x & 31, sw = lane / G;
    const bool active = (sw < P) && (sw < it.rep_count);
    const int seg = sw < P ? lane - sw * G : 0;
    const int kglob = it.rep_begin + sw + 1;
    const uint32_t key = (p.flags & BD_FLAG_IDENTICAL_NOISE) ? 0u : (uint32_t)kglob;
    const LaneCtx lc = make_lane(seg, G, L, lane, nb, active, key, (uint32_t)it.chain + p.chain_base);
    const int64_t w = a.w_batch0 + blockIdx.y;
    const int64_t tw = w * p.S;
    const int64_t row = a.state_bonds * 3;                  // one step of repbuf
    T* rb = reinterpret_cast<T*>(a.repbuf) + (int64_t)blockIdx.y * (p.S + 1) * row +
            (ch.state_off + (int64_t)kglob * nb) * 3;

    // forward: spawn from the parent at tw, S steps, every state kept
    {
        uint4* tab = tab_all[threadIdx.x >> 5];
        for (int b = lane; b < G * L; b += 32)
            tab[b] = PhiloxSplit::bead_part((uint32_t)b, (uint32_t)it.chain + p.chain_base, p.rk0, p.rk1);
        __syncwarp();
        StepConst<T, FAST> k;
        k.load(ch, p);
        T qx[L], qy[L], qz[L];
        load_bonds<T, L>(qx, qy, qz,
                         reinterpret_cast<const T*>(a.segbuf) + ((tw - a.seg_t0) * p.M + ch.spr_off) * 3, lc);
        store_bonds<T, L>(qx, qy, qz, rb, lc);
#pragma unroll 1
        for (int s = 0; s < p.S; ++s) {
            step_bonds<T, L, FAST, true>(qx, qy, qz, lc, k, (uint32_t)(tw + s), p, tab);
            store_bonds<T, L>(qx, qy, qz, rb + (int64_t)(s + 1) * row, lc);
        }
    }

    // backward
    AdjConst<T> k;
    k.load(ch, ac, p);
    GradAcc<T> ga;
    ga.init();
    T lx[L], ly[L], lz[L];
    {
        const T* q = rb + (int64_t)p.S * row;
        const double* Gw = a.G + (w - a.w_lo) * p.M + ch.spr_off;
        const double invR = 1.0 / (double)ch.R;
#pragma unroll
        for (int j = 0; j < L; ++j) {
            lx[j] = ly[j] = lz[j] = T(0);
            if (j < lc.nv) {
                const int i = lc.bead0 + j;
                const T gi = (T)(Gw[i] * invR);
                const T qx = q[3 * i + 0], qy = q[3 * i + 1], qz = q[3 * i + 2];
                const T q2 = fma(qx, qx, fma(qy, qy, qz * qz));
                const T qn = sqrt(q2);
                SpringD<T> sd;
                sd.at(q2, k.H, k.Hinvb, k.smin);
                // grad f = (c / |Q| + 2 (dc/d|Q|^2) |Q|) Q; df/dtheta = (dc/dtheta) |Q|
                const T fac = qn > T(0) ? gi * (sd.c / qn + T(2) * sd.dcq * qn) : T(0);
                lx[j] = fac * qx; ly[j] = fac * qy; lz[j] = fac * qz;
                ga.part[1] = fma(gi * sd.dcb, qn, ga.part[1]);
                ga.part[2] = fma(gi * sd.dcH, qn, ga.part[2]);
            }
        }
    }
    // states are loaded one step ahead of the sweep that uses them
    T qx[L], qy[L], qz[L];
    load_lane<T, L>(rb + (int64_t)(p.S - 1) * row, lc, qx, qy, qz);
#pragma unroll 1
    for (int s = p.S - 1; s >= 0; --s) {
        T nx[L], ny[L], nz[L];
        load_lane<T, L>(rb + (int64_t)(s > 0 ? s - 1 : 0) * row, lc, nx, ny, nz);
        adjoint_step<T, L>(qx, qy, qz, lx, ly, lz, lc, k, ga.part);
        ga.tick();
#pragma unroll
        for (int j = 0; j < L; ++j) { qx[j] = nx[j]; qy[j] = ny[j]; qz[j] = nz[j]; }
    }
    ga.fold();

    // mu_w of this item: float64 sum over its replicas, in replica order, by
    // the lanes of the first replica
    const int src0 = sw < P ? seg : lane;
    double* mrow = a.mu + ((w - a.mu_w0) * a.mu_stride + ac.part_off + (int64_t)it.group * nb) * 3;
#pragma unroll
    for (int j = 0; j < L; ++j) {
        double sx = 0.0, sy = 0.0, sz = 0.0;
        for (int s2 = 0; s2 < P; ++s2) {
            const int src = sw < P ? s2 * G + src0 : lane;
            const T vx = shfl(lx[j], src), vy = shfl(ly[j], src), vz = shfl(lz[j], src);
            if (s2 < it.rep_count) { sx += (double)vx; sy += (double)vy; sz += (double)vz; }
        }
        if (sw == 0 && j < lc.nv) {
            const int i = lc.bead0 + j;
            mrow[3 * i + 0] = sx; mrow[3 * i + 1] = sy; mrow[3 * i + 2] = sz;
        }
    }
    // every lane of the item belongs to one chain: warp sum, one atomic each
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        double x = ga.sum[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) atomicAdd(a.grad + 3 * it.chain + j, x);
    }
}

// ---------------------------------------------------------------------------
// Parent backward over steps [t0, t0 + n_steps): lambda from lamP, adjoint
// steps down to t0, adding mu_w where a window of the objective starts;
// lambda back to lamP.
// ---------------------------------------------------------------------------
template <typename T, int L>
__global__ void __launch_bounds__(kAdjThreads) adj_parent_backward_kernel(const AdjParams a)
{
    const StepParams& p = a.sp;
    ParentLane pl;
    if (!parent_lane<L>(p, pl)) return;
    const LaneCtx& lc = pl.lc;
    const ChainDev ch = p.chains[pl.chain];
    const AdjChain ac = a.adj[pl.chain];
    const int nb = ch.N - 1;
    AdjConst<T> k;
    k.load(ch, ac, p);
    const T* seg = reinterpret_cast<const T*>(a.segbuf) + ch.spr_off * 3;
    T* lp = reinterpret_cast<T*>(a.lamP) + ch.spr_off * 3;
    GradAcc<T> ga;
    ga.init();
    T lx[L], ly[L], lz[L];
    load_bonds<T, L>(lx, ly, lz, lp, lc);
    // states are loaded one step ahead of the sweep that uses them
    T qx[L], qy[L], qz[L];
    if (a.n_steps > 0)
        load_lane<T, L>(seg + (a.t0 + a.n_steps - 1 - a.seg_t0) * p.M * 3, lc, qx, qy, qz);
#pragma unroll 1
    for (int s = a.n_steps - 1; s >= 0; --s) {
        const int64_t t = a.t0 + s;
        T nx[L], ny[L], nz[L];
        load_lane<T, L>(seg + ((s > 0 ? t - 1 : t) - a.seg_t0) * p.M * 3, lc, nx, ny, nz);
        adjoint_step<T, L>(qx, qy, qz, lx, ly, lz, lc, k, ga.part);
        ga.tick();
#pragma unroll
        for (int j = 0; j < L; ++j) { qx[j] = nx[j]; qy[j] = ny[j]; qz[j] = nz[j]; }
        const int64_t w = t / p.S;
        if (t == w * p.S && w >= a.w_lo && w < a.w_hi) {
            const double* mrow = a.mu + ((w - a.mu_w0) * a.mu_stride + ac.part_off) * 3;
#pragma unroll
            for (int j = 0; j < L; ++j) {
                if (j < lc.nv) {
                    const int i = lc.bead0 + j;
                    double sx = 0.0, sy = 0.0, sz = 0.0;
                    for (int g = 0; g < ac.n_groups; ++g) {
                        const double* e = mrow + ((int64_t)g * nb + i) * 3;
                        sx += e[0]; sy += e[1]; sz += e[2];
                    }
                    lx[j] = (T)((double)lx[j] + sx);
                    ly[j] = (T)((double)ly[j] + sy);
                    lz[j] = (T)((double)lz[j] + sz);
                }
            }
        }
    }
    ga.fold();
    store_bonds<T, L>(lx, ly, lz, lp, lc);
    // a warp may hold several chains: one atomic per lane with work
    if (lc.nv > 0) {
#pragma unroll
        for (int j = 0; j < 3; ++j) atomicAdd(a.grad + 3 * pl.chain + j, ga.sum[j]);
    }
}

}  // namespace bdra
