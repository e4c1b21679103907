// C ABI of the replica-averaged Brownian-dynamics library (include/bdra.h):
// configuration checks, launch planning, device state, and the stream-ordered
// driving of the parent / replica kernels and the support kernels.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "bd_launch.h"
#include "bd_support.h"

using namespace bdra;

namespace {

struct VarClass {      // one persistent replica launch: the work items of one step variant
    int variant;
    int item_begin, item_count;
    int grid, threads;
    size_t smem;       // dynamic shared memory per CTA
};
struct ParClass {      // one parent-kernel launch: the parent warps of one tile
    int L, threads, grid;
    int warp_begin, warp_count;
    bool lj;           // collapsed chains (harmonic springs, pair forces)
    bool hi;           // hydrodynamic interaction: one CTA per parent
    size_t smem;
};
constexpr int kParentLJKey = 1000;   // planner key offset of the collapsed-chain parents
constexpr int kParentHIKey = 2000;   // planner key of the parents with hydrodynamic interaction

struct AdjClass {      // one adjoint replica-window launch: the work items of one tile
    int L;
    int item_begin, item_count;
};

}  // namespace

struct bd_ctx {
    bd_config cfg;
    std::vector<bd_chain_desc> chains;
    cudaStream_t stream = nullptr;
    int device = 0;
    bool f64 = false;
    size_t tsize = 4;
    int64_t M = 0, n_beads = 0, n_slot_beads = 0, state_bonds = 0, part_stride = 0;
    int64_t step = 0, windows_detected = 0, chunk_windows = 0;
    std::vector<ChainDev> h_chains;
    std::vector<ItemDev> h_items;
    std::vector<int32_t> h_parent_items;
    std::vector<ParentWarp> h_parent_warps;
    std::vector<VarClass> var_classes;
    std::vector<ParClass> par_classes;
    double var_cost[kVariantCodes];     // issue cost per warp-step of each variant
    uint32_t rk0[10], rk1[10];

    ChainDev* d_chains = nullptr;
    ItemDev* d_items = nullptr;
    int32_t* d_parent_items = nullptr;
    ParentWarp* d_parent_warps = nullptr;
    int32_t* d_spring_chain = nullptr;
    int64_t* d_pair_parent = nullptr;   // [n_chains + 1] prefix of 1 per chain
    int64_t* d_pair_all = nullptr;      // [n_chains + 1] prefix of R + 1 per chain
    void* d_state = nullptr;
    void* d_snap = nullptr;
    double* d_part = nullptr;           // [part_ring][part_stride] per-group partial sums
    double* d_rsf = nullptr;            // [max_windows][M] replica-averaged force history
    int32_t part_ring = 0;              // windows the snapshot and partial rings hold (one chunk's + 1)
    // conformation diagnostics of Eq. 5 (BD_FLAG_CONFORMATION)
    bool conf = false;
    int64_t n_rep = 0, bpart_stride = 0;
    int32_t* d_bead_chain = nullptr;    // [sum N] chain of each bead
    double* d_dbar = nullptr;           // [max_windows][sum R][3]
    double* d_dpart = nullptr;          // [part_ring][bpart_stride][3]
    double* d_dbead = nullptr;          // [max_windows][sum N][3]
    double* d_rgz = nullptr;            // [max_windows][n_chains]
    double* d_tsf = nullptr;
    double* d_tsf_acc = nullptr;
    double* d_lam = nullptr;
    int64_t* d_first_thr = nullptr;
    int64_t* d_first_bell = nullptr;
    double* d_exp1 = nullptr;
    unsigned long long* d_overext = nullptr;
    int32_t* d_dev_err = nullptr;       // error bits set by kernels whose bounded waits gave up
    int64_t* d_evt_scratch = nullptr;
    int32_t* d_queue = nullptr;         // one work-item counter per variant launch
    // the step chunk as a CUDA graph: queue reset, parent kernels, one
    // persistent replica kernel per variant (parallel branches), and three
    // event records (start, after the parents, after the replicas)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<cudaGraphNode_t> par_nodes, rep_nodes;
    cudaGraphNode_t ev_nodes[3] = {nullptr, nullptr, nullptr};
    cudaGraphNode_t fold_node = nullptr;     // partial sums -> RSF history, after the replicas
    cudaEvent_t idle_ev[3] = {nullptr, nullptr, nullptr};
    int n_sm = 0;
    void* d_io = nullptr;
    size_t io_bytes = 0;
    size_t bytes = 0;
    std::vector<void*> allocs;
    std::string err;
    int64_t launches = 0;
    bool timing = false;
    double timed_ms[2] = {0.0, 0.0};   // accumulated parent / replica time
    int64_t timed_n[2] = {0, 0};
    // adjoint (cfg.checkpoint_steps > 0): parent checkpoints every K steps
    // from `origin` (the step of bd_create / bd_set_positions), the adjoint
    // plan, and work buffers allocated by the first bd_adjoint
    int64_t origin = 0;
    void* d_ckpt = nullptr;
    int64_t n_ckpt = 0;
    std::vector<AdjChain> h_adj;
    std::vector<ItemDev> h_adj_items;
    std::vector<AdjClass> adj_classes;
    int64_t adj_stride = 0, rep_batch = 0;
    AdjChain* d_adj = nullptr;
    ItemDev* d_adj_items = nullptr;
    void* d_seg[2] = {nullptr, nullptr};    // parent segments, alternating
    void* d_repbuf = nullptr;
    void* d_lamP = nullptr;
    double* d_mu[2] = {nullptr, nullptr};   // window sensitivities, alternating batches
    // the parent's backward sweeps run on their own stream, overlapping the
    // next batch of replica windows; events order the shared buffers
    cudaStream_t adj_stream = nullptr;
    cudaEvent_t ev_init = nullptr, ev_done = nullptr;
    cudaEvent_t ev_win[2] = {nullptr, nullptr}, ev_mu_free[2] = {nullptr, nullptr};
    cudaEvent_t ev_seg_free[2] = {nullptr, nullptr};
    double* d_gls = nullptr;
    double* d_grad = nullptr;
    double* d_G = nullptr;
    size_t G_bytes = 0;
};

namespace {

bd_status fail(bd_ctx* ctx, bd_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    return s;
}

#define BD_CUDA(ctx, call)                                                                    \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            cudaGetLastError();                                                               \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? BD_E_OOM : BD_E_CUDA,          \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,     \
                        __LINE__);                                                            \
        }                                                                                     \
    } while (0)

bd_status dalloc(bd_ctx* ctx, void** p, size_t n)
{
    *p = nullptr;
    if (n == 0) n = 16;
    cudaError_t e = cudaMalloc(p, n);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(ctx, BD_E_OOM, "cudaMalloc of %zu bytes failed: %s", n, cudaGetErrorString(e));
    }
    ctx->allocs.push_back(*p);
    ctx->bytes += n;
    return BD_OK;
}

void dfree(bd_ctx* ctx, void* p, size_t n)
{
    if (!p) return;
    cudaFree(p);
    auto it = std::find(ctx->allocs.begin(), ctx->allocs.end(), p);
    if (it != ctx->allocs.end()) ctx->allocs.erase(it);
    ctx->bytes -= n;
}

bool is_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bd_status ensure_io(bd_ctx* ctx, size_t n)
{
    if (ctx->io_bytes >= n) return BD_OK;
    if (ctx->d_io) {
        BD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        cudaFree(ctx->d_io);
        auto it = std::find(ctx->allocs.begin(), ctx->allocs.end(), ctx->d_io);
        if (it != ctx->allocs.end()) ctx->allocs.erase(it);
        ctx->bytes -= ctx->io_bytes;
        ctx->d_io = nullptr;
        ctx->io_bytes = 0;
    }
    bd_status s = dalloc(ctx, &ctx->d_io, n);
    if (s == BD_OK) ctx->io_bytes = n;
    return s;
}

// Philox round keys: key + r * (Weyl constants).
void round_keys(uint64_t seed, uint32_t* rk0, uint32_t* rk1)
{
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        rk0[r] = k0; rk1[r] = k1;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
}

// ---------------------------------------------------------------------------
// Launch planning (the autotuner's cost model). For a chain of N beads and R
// replicas and each tile size L (springs per lane): G = ceil(N / L) lanes per
// slot, P = 32 / G slots per warp, at most Wmax warps per CTA; the replicas
// split into the fewest groups that fit, and the cost is the lane-steps issued
// per useful bead-step, with a fixed per-lane overhead for the halo exchange.
// ---------------------------------------------------------------------------
struct VariantChoice { int variant, per_warp, groups; double cost; };

// Default issue cost per warp-step (lane-instructions): one replica per lane
// ~100 per spring plus the halo exchange; two replicas per lane ~110 per
// spring pair (packed float32 arithmetic, one Philox call for the pair's
// noise, per-normal special functions). bd_autotune replaces these with
// measured times.
double default_variant_cost(int v)
{
    const int L = variant_tile(v);
    if (variant_lj(v)) return 1000.0 * L;      // pair forces: work per lane grows with its beads
    return variant_paired(v) ? 110.0 * L + 60.0 : 100.0 * L + 40.0;
}

// Warp work items of a chain with R replicas, at most per_warp replicas an
// item, and how they split. Replicas 2j - 1 and 2j form a noise pair (one
// generator output, two halves). With two replicas per lane (variant v
// paired) the split is in whole pairs, so that every item starts at an even
// offset and each lane holds one pair (one generator call for both). With
// one replica per lane and several replicas a warp, the odd replicas and the
// even ones go to separate items (stride 2), so that all lanes of a warp
// draw the same half (no divergence). Each set splits as evenly as its
// items allow.
int item_count(int R, int per_warp, int v)
{
    if (variant_paired(v) || per_warp == 1) return (R + per_warp - 1) / per_warp;
    const int odd = (R + 1) / 2, even = R / 2;
    return (odd + per_warp - 1) / per_warp + (even + per_warp - 1) / per_warp;
}

void split_run(int c, int& g, int n, int groups, int first, int stride, int unit, int v,
               std::vector<ItemDev>& items)
{
    // n replicas first, first + stride, ..., in `groups` items (unit: whole pairs)
    const int units = (n + unit - 1) / unit;
    int done = 0;
    for (int k = 0; k < groups; ++k) {
        const int uk = units / groups + (k < units % groups ? 1 : 0);
        const int cnt = std::min(uk * unit, n - done);
        items.push_back(ItemDev{c, g++, first + stride * done, cnt, v, stride});
        done += cnt;
    }
}

// Work-item order of the persistent launches: by variant, and within one the
// items whose replicas draw the first noise half before those that draw the
// second (a one-replica-per-lane item of one half runs its own copy of the
// step code, and keeping the halves apart keeps one copy in the instruction
// cache at a time), each in chain order.
void order_items(std::vector<ItemDev>& items)
{
    auto half_of = [](const ItemDev& it) {
        return (it.stride == 2 || it.rep_count == 1) ? (int)(((it.rep_begin + 1) & 1) == 0) : 0;
    };
    std::stable_sort(items.begin(), items.end(), [&](const ItemDev& x, const ItemDev& y) {
        return x.variant != y.variant ? x.variant < y.variant : half_of(x) < half_of(y);
    });
}

// The one-replica-per-lane kernels compile one noise half per item, so the
// items built here must be single replicas or stride-2 runs (a mixed item
// would draw the wrong half for some of its replicas).
void split_replicas(int c, int R, int per_warp, int v, std::vector<ItemDev>& items)
{
    int g = 0;
    if (variant_paired(v)) {
        split_run(c, g, R, (R + per_warp - 1) / per_warp, 0, 1, 2, v, items);
    } else if (per_warp == 1) {
        split_run(c, g, R, R, 0, 1, 1, v, items);
    } else {
        const int odd = (R + 1) / 2, even = R / 2;
        split_run(c, g, odd, (odd + per_warp - 1) / per_warp, 0, 2, 1, v, items);
        split_run(c, g, even, (even + per_warp - 1) / per_warp, 1, 2, 1, v, items);
    }
}

// The step variant for a chain: a warp holds P = 32 / ceil(N / L) replicas
// (2P with two replicas per lane); the chain needs ceil(R / per_warp) warp
// items, and the cost is their issue work per useful bead-step. Collapsed
// chains (harmonic springs) take the collapsed-chain variants, the others
// the rest; the tile and layout hints apply to the latter.
VariantChoice choose_variant(const bd_ctx* ctx, int N, int R, bool collapsed, bool hi)
{
    const bd_config& cfg = ctx->cfg;
    if (hi) return {kHIBase + (N > kHISmallBeadsHost ? 1 : 0), 1, R, 0.0};   // one CTA per replica
    const int* vars = ctx->f64 ? kVariantsF64 : kVariantsF32;
    const int nv = ctx->f64 ? kNumVariantsF64 : kNumVariantsF32;
    VariantChoice best{0, 0, 0, 1e300};
    for (int t = 0; t < nv; ++t) {
        const int v = vars[t];
        const bool paired = variant_paired(v);
        const int L = variant_tile(v);
        if (variant_lj(v) != collapsed) continue;
        if (!collapsed) {
            if (cfg.lanes_hint && L != cfg.lanes_hint) continue;
            if (cfg.layout_hint == 1 && paired) continue;
            if (cfg.layout_hint == 2 && !paired) continue;
        }
        const int G = (N + L - 1) / L;
        if (G > 32) continue;
        const int per_warp = (paired ? 2 : 1) * (32 / G);
        const int groups = item_count(R, per_warp, v);
        const double cost = groups * ctx->var_cost[v] / ((double)R * N);
        if (cost < best.cost - 1e-12) best = {v, per_warp, groups, cost};
    }
    return best;
}

// The parent kernel is latency-bound (one slot per chain): the smallest tile
// that fits a chain in one warp gives the shortest step.
int choose_parent_tile(int N)
{
    for (int t = 0; t < kNumTiles; ++t)
        if ((N + kTiles[t] - 1) / kTiles[t] <= 32) return kTiles[t];
    return 0;
}

bd_status validate(bd_ctx* ctx, const bd_config* cfg)
{
    if (!cfg) return fail(ctx, BD_E_INVALID, "cfg is NULL");
    if (cfg->n_chains < 1) return fail(ctx, BD_E_INVALID, "n_chains must be >= 1");
    if (!cfg->chains) return fail(ctx, BD_E_INVALID, "chains is NULL");
    if (cfg->window_steps < 1) return fail(ctx, BD_E_INVALID, "window_steps must be >= 1");
    if (!(cfg->dt > 0) || !std::isfinite(cfg->dt)) return fail(ctx, BD_E_INVALID, "dt must be > 0");
    if (cfg->precision != BD_PREC_FP32 && cfg->precision != BD_PREC_FP64)
        return fail(ctx, BD_E_INVALID, "unknown precision %d", cfg->precision);
    if (cfg->max_windows < 0) return fail(ctx, BD_E_INVALID, "max_windows must be >= 0");
    if (!(cfg->s_min > 0 && cfg->s_min < 1)) return fail(ctx, BD_E_INVALID, "s_min must be in (0, 1)");
    if ((cfg->thr_mask & ~7) || (cfg->bell_mask & ~7))
        return fail(ctx, BD_E_INVALID, "criterion masks use bits 0..2 only");
    if (cfg->flags & ~(BD_FLAG_IDENTICAL_NOISE | BD_FLAG_CONFORMATION | BD_FLAG_TEST_TC_STALL))
        return fail(ctx, BD_E_INVALID, "unknown flags");
    if (cfg->checkpoint_steps < 0 || (cfg->checkpoint_steps > 0 && cfg->checkpoint_steps % cfg->window_steps))
        return fail(ctx, BD_E_INVALID, "checkpoint_steps must be 0 or a positive multiple of window_steps");
    if (cfg->chain_id_base < 0 || (int64_t)cfg->chain_id_base + cfg->n_chains - 1 > INT32_MAX)
        return fail(ctx, BD_E_INVALID, "chain_id_base must be >= 0 with chain_id_base + n_chains - 1 <= 2^31 - 1");
    if (cfg->layout_hint < 0 || cfg->layout_hint > 2)
        return fail(ctx, BD_E_INVALID, "layout_hint must be 0, 1 or 2");
    if (cfg->layout_hint == 2 && cfg->precision != BD_PREC_FP32)
        return fail(ctx, BD_E_INVALID, "two replicas per lane needs float32 integration");
    if (cfg->lanes_hint) {
        const bool f64 = cfg->precision == BD_PREC_FP64;
        const int* vars = f64 ? kVariantsF64 : kVariantsF32;
        const int nv = f64 ? kNumVariantsF64 : kNumVariantsF32;
        bool ok = false;
        for (int t = 0; t < nv; ++t) {
            const bool paired = variant_paired(vars[t]);
            if (variant_lj(vars[t]) || variant_tile(vars[t]) != cfg->lanes_hint) continue;   // FENE/Hooke variants
            if ((cfg->layout_hint == 1 && paired) || (cfg->layout_hint == 2 && !paired)) continue;
            ok = true;
        }
        if (!ok)
            return fail(ctx, BD_E_INVALID, "lanes_hint %d is not a compiled step variant for this layout",
                        cfg->lanes_hint);
    }
    for (int c = 0; c < cfg->n_chains; ++c) {
        const bd_chain_desc& d = cfg->chains[c];
        if (d.n_beads < 2 || d.n_beads > 512)
            return fail(ctx, BD_E_INVALID, "chain %d: n_beads %d outside [2, 512]", c, d.n_beads);
        if (d.n_replicas < 1 || d.n_replicas > 4096)
            return fail(ctx, BD_E_INVALID, "chain %d: n_replicas %d outside [1, 4096]", c, d.n_replicas);
        const bool rest_law = d.spring == BD_SPRING_HARMONIC || d.spring == BD_SPRING_VWF;
        if (d.spring != BD_SPRING_HOOKE && d.spring != BD_SPRING_FENE && !rest_law)
            return fail(ctx, BD_E_INVALID, "chain %d: unknown spring law %d", c, d.spring);
        if (rest_law && (!(d.r0 >= 0) || !std::isfinite(d.r0)))
            return fail(ctx, BD_E_INVALID, "chain %d: harmonic rest length must be >= 0", c);
        if (!(d.lj_u >= 0) || !std::isfinite(d.lj_u))
            return fail(ctx, BD_E_INVALID, "chain %d: lj_u must be >= 0", c);
        if (d.spring == BD_SPRING_VWF &&
            (!(d.vwf_fa >= 0) || !(d.vwf_fb >= 0) || !(d.vwf_xmax > 0) || !std::isfinite(d.vwf_fa) ||
             !std::isfinite(d.vwf_fb) || !std::isfinite(d.vwf_xmax)))
            return fail(ctx, BD_E_INVALID, "chain %d: vWF needs vwf_fa, vwf_fb >= 0 and vwf_xmax > 0", c);
        if (d.lj_u > 0 && (!rest_law || !(d.lj_sigma > 0) || !std::isfinite(d.lj_sigma)))
            return fail(ctx, BD_E_INVALID, "chain %d: Lennard-Jones needs the harmonic law and lj_sigma > 0", c);
        if (rest_law && cfg->checkpoint_steps > 0)
            return fail(ctx, BD_E_INVALID, "chain %d: the adjoint supports Hooke and FENE chains only", c);
        if (!(d.hi_a >= 0) || !std::isfinite(d.hi_a))
            return fail(ctx, BD_E_INVALID, "chain %d: hi_a must be >= 0", c);
        if (d.hi_a > 0) {
            if (d.n_beads > kHIMaxBeadsHost)
                return fail(ctx, BD_E_INVALID, "chain %d: hydrodynamic interaction needs n_beads <= %d",
                            c, kHIMaxBeadsHost);
            if (cfg->checkpoint_steps > 0)
                return fail(ctx, BD_E_INVALID, "chain %d: no adjoint with hydrodynamic interaction", c);
        }
        if (d.flow < BD_FLOW_NONE || d.flow > BD_FLOW_PLANAR)
            return fail(ctx, BD_E_INVALID, "chain %d: unknown flow %d", c, d.flow);
        if (!(d.H > 0) || !std::isfinite(d.H)) return fail(ctx, BD_E_INVALID, "chain %d: H must be > 0", c);
        if (d.spring == BD_SPRING_FENE && (!(d.b > 0) || !std::isfinite(d.b)))
            return fail(ctx, BD_E_INVALID, "chain %d: FENE b must be > 0", c);
        if (!std::isfinite(d.rate)) return fail(ctx, BD_E_INVALID, "chain %d: rate not finite", c);
    }
    if (cfg->lanes_hint) {
        for (int c = 0; c < cfg->n_chains; ++c)
            if (cfg->chains[c].spring != BD_SPRING_HARMONIC && cfg->chains[c].spring != BD_SPRING_VWF &&
                !(cfg->chains[c].hi_a > 0) &&
                (cfg->chains[c].n_beads + cfg->lanes_hint - 1) / cfg->lanes_hint > 32)
                return fail(ctx, BD_E_INVALID, "lanes_hint %d too small for chain %d (N=%d)",
                            cfg->lanes_hint, c, cfg->chains[c].n_beads);
    }
    return BD_OK;
}

bd_status plan(bd_ctx* ctx)
{
    const bd_config& cfg = ctx->cfg;
    const int C = cfg.n_chains;
    ctx->h_chains.resize(C);
    int64_t bead = 0, slot_bead = 0, bond = 0, spr = 0, part = 0, rep = 0, bpart = 0;
    std::vector<ItemDev> items;
    // ((L + kParentLJKey if collapsed, G), chain): one parent launch per key
    std::vector<std::pair<std::pair<int, int>, int>> par;
    for (int c = 0; c < C; ++c) {
        const bd_chain_desc& d = ctx->chains[c];
        ChainDev& h = ctx->h_chains[c];
        const bool collapsed = d.spring == BD_SPRING_HARMONIC || d.spring == BD_SPRING_VWF;
        const bool hi = d.hi_a > 0;
        const VariantChoice vc = choose_variant(ctx, d.n_beads, d.n_replicas, collapsed, hi);
        if (!vc.variant)
            return fail(ctx, BD_E_INVALID, "chain %d: no step variant fits N=%d", c, d.n_beads);
        h.N = d.n_beads; h.R = d.n_replicas; h.n_groups = vc.groups; h.spring = d.spring;
        h.hi_a = d.hi_a;
        h.bead_off = bead; h.slot_bead_off = slot_bead; h.state_off = bond;
        h.spr_off = spr; h.part_off = part;
        h.rep_off = rep; h.bpart_off = bpart;
        h.H = d.H;
        h.Hinvb = d.spring == BD_SPRING_FENE ? d.H / d.b : 0.0;
        h.kxx = h.kyy = h.kzz = h.kxz = 0.0;
        switch (d.flow) {
        case BD_FLOW_SHEAR: h.kxz = d.rate; break;
        case BD_FLOW_UNIAXIAL: h.kxx = d.rate; h.kyy = -0.5 * d.rate; h.kzz = -0.5 * d.rate; break;
        case BD_FLOW_PLANAR: h.kxx = d.rate; h.kyy = -d.rate; break;
        default: break;
        }
        h.f_c = d.f_c; h.k0 = d.k0; h.dx = d.dx;
        h.r0 = collapsed ? d.r0 : 0.0;
        h.vwf_fa = d.spring == BD_SPRING_VWF ? d.vwf_fa : 0.0;
        h.vwf_fb = d.spring == BD_SPRING_VWF ? d.vwf_fb : 0.0;
        h.vwf_ix2 = d.spring == BD_SPRING_VWF ? 1.0 / (d.vwf_xmax * d.vwf_xmax) : 0.0;
        h.lj_u = d.lj_u;
        h.lj_s2 = d.lj_sigma * d.lj_sigma;
        // float32 step constants, rounded as (float)(double expression);
        // sqrt(2 D dt) carries the sign of the fast float normals (-1)
        h.f32[0] = (float)h.H;
        h.f32[1] = (float)h.Hinvb;
        h.f32[2] = (float)(0.25 * cfg.dt);
        h.f32[3] = (float)std::sqrt(0.5 * cfg.dt) * -1.0f;
        h.f32[4] = (float)(h.kxx * cfg.dt);
        h.f32[5] = (float)(h.kyy * cfg.dt);
        h.f32[6] = (float)(h.kzz * cfg.dt);
        h.f32[7] = (float)(h.kxz * cfg.dt);
        h.f32[8] = (float)cfg.s_min;
        h.f32_pad = 0.0f;
        const int nb = d.n_beads - 1;
        // warp items: replicas split as evenly as the warp capacity allows
        split_replicas(c, d.n_replicas, vc.per_warp, vc.variant, items);
        if (hi) {
            par.push_back({{kParentHIKey + (d.n_beads > kHISmallBeadsHost ? 1 : 0), 1}, c});
        } else {
            const int Lp = choose_parent_tile(d.n_beads);
            par.push_back({{Lp + (collapsed ? kParentLJKey : 0), (d.n_beads + Lp - 1) / Lp}, c});
        }
        bead += d.n_beads;
        slot_bead += (int64_t)(d.n_replicas + 1) * d.n_beads;
        bond += (int64_t)(d.n_replicas + 1) * nb;
        spr += nb;
        part += (int64_t)vc.groups * nb;
        rep += d.n_replicas;
        bpart += (int64_t)vc.groups * d.n_beads;
    }
    ctx->n_rep = rep;
    ctx->bpart_stride = bpart;
    ctx->n_beads = bead; ctx->n_slot_beads = slot_bead; ctx->state_bonds = bond;
    ctx->M = spr; ctx->part_stride = part;

    // persistent replica launches: one per variant, items ordered by noise half
    order_items(items);
    ctx->h_items = items;
    ctx->var_classes.clear();
    const int threads = ctx->f64 ? persist_threads_f64() : persist_threads_f32();
    for (size_t k = 0; k < items.size(); ++k) {
        if (ctx->var_classes.empty() || ctx->var_classes.back().variant != items[k].variant)
            ctx->var_classes.push_back(VarClass{items[k].variant, (int)k, 0, 0, threads, 0});
        ctx->var_classes.back().item_count++;
    }
    for (VarClass& vc : ctx->var_classes) {
        if (variant_hi(vc.variant)) {          // one CTA per replica
            cudaError_t e = ctx->f64 ? hi_prepare_f64() : hi_prepare_f32();
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(ctx, BD_E_CUDA, "hydrodynamic-interaction kernels: %s", cudaGetErrorString(e));
            }
            vc.threads = ctx->f64 ? hi_threads_f64(vc.variant == kHIBase) : hi_threads_f32(vc.variant == kHIBase);
            vc.grid = vc.item_count;
            vc.smem = ctx->f64 ? hi_smem_f64(vc.variant == kHIBase) : hi_smem_f32(vc.variant == kHIBase);
            continue;
        }
        vc.smem = ctx->f64 ? persist_smem_f64(vc.variant) : persist_smem_f32(vc.variant);
        int per_sm = 1;
        cudaError_t e = ctx->f64 ? persist_blocks_per_sm_f64(vc.variant, ctx->conf, &per_sm)
                                 : persist_blocks_per_sm_f32(vc.variant, ctx->conf, &per_sm);
        if (e != cudaSuccess || per_sm < 1) {
            cudaGetLastError();
            return fail(ctx, BD_E_CUDA, "occupancy of variant %d: %s", vc.variant, cudaGetErrorString(e));
        }
        const int warps = threads / 32;
        const int need = (vc.item_count + warps - 1) / warps;
        vc.grid = std::max(1, std::min(need, per_sm * ctx->n_sm));
    }
    // parent launches: one per tile; warps pack parents of equal lane count
    std::stable_sort(par.begin(), par.end());
    ctx->h_parent_items.clear();
    ctx->h_parent_warps.clear();
    ctx->par_classes.clear();
    for (size_t k = 0; k < par.size();) {
        const int key = par[k].first.first, G = par[k].first.second;
        const bool hi = key >= kParentHIKey;
        const int P = hi ? 1 : 32 / G;           // one CTA per parent with hydrodynamic interaction
        const int L = hi ? key - kParentHIKey : key % kParentLJKey;   // hi: 0 small, 1 large chains
        const bool lj = !hi && key >= kParentLJKey;
        if (ctx->par_classes.empty() || ctx->par_classes.back().L != L || ctx->par_classes.back().lj != lj ||
            ctx->par_classes.back().hi != hi)
            ctx->par_classes.push_back(ParClass{L, hi ? (ctx->f64 ? hi_threads_f64(L == 0) : hi_threads_f32(L == 0))
                                                      : kParentThreads, 0,
                                                (int)ctx->h_parent_warps.size(), 0, lj, hi,
                                                hi ? (ctx->f64 ? hi_smem_f64(L == 0) : hi_smem_f32(L == 0)) : 0});
        size_t e = k;
        while (e < par.size() && par[e].first == par[k].first) ++e;
        for (size_t j = k; j < e; j += P) {
            const int cnt = (int)std::min<size_t>(P, e - j);
            ctx->h_parent_warps.push_back(ParentWarp{(int32_t)ctx->h_parent_items.size(), cnt, G, 0});
            for (int s = 0; s < cnt; ++s) ctx->h_parent_items.push_back(par[j + s].second);
            ctx->par_classes.back().warp_count++;
        }
        k = e;
    }
    for (ParClass& pc : ctx->par_classes) {
        const int per_cta = pc.hi ? 1 : pc.threads / 32;
        pc.grid = (pc.warp_count + per_cta - 1) / per_cta;
    }
    // snapshot chunk: up to 64 windows, capped at ~512 MB
    const int64_t per_window = ctx->M * 3 * (int64_t)ctx->tsize;
    ctx->chunk_windows = std::max<int64_t>(1, std::min<int64_t>(64, (512ll << 20) / std::max<int64_t>(per_window, 1)));
    return BD_OK;
}

StepParams base_params(const bd_ctx* ctx)
{
    StepParams p;
    std::memset(&p, 0, sizeof(p));
    p.chains = ctx->d_chains;
    p.items = ctx->d_items;
    p.parent_items = ctx->d_parent_items;
    p.state = ctx->d_state;
    p.snap = ctx->d_snap;
    p.part_hist = ctx->d_part;
    p.win_ring = ctx->part_ring;
    p.dbar = ctx->d_dbar;
    p.dbead_part = ctx->d_dpart;
    p.rgz = ctx->d_rgz;
    p.n_rep = ctx->n_rep;
    p.bpart_stride = ctx->bpart_stride;
    p.n_chains = ctx->cfg.n_chains;
    p.chain_base = (uint32_t)ctx->cfg.chain_id_base;
    p.tsf_hist = ctx->d_tsf;
    p.tsf_acc = ctx->d_tsf_acc;
    p.lam = ctx->d_lam;
    p.first_thr = ctx->d_first_thr;
    p.first_bell = ctx->d_first_bell;
    p.exp1 = ctx->d_exp1;
    p.overext = ctx->d_overext;
    p.dev_err = ctx->d_dev_err;
    p.part_stride = ctx->part_stride;
    p.M = ctx->M;
    p.dt = ctx->cfg.dt;
    p.s_min = ctx->cfg.s_min;
    p.S = ctx->cfg.window_steps;
    p.flags = ctx->cfg.flags;
    p.thr_mask = ctx->cfg.thr_mask;
    p.bell_mask = ctx->cfg.bell_mask;
    p.key0 = (uint32_t)ctx->cfg.seed;
    p.key1 = (uint32_t)(ctx->cfg.seed >> 32);
    std::memcpy(p.rk0, ctx->rk0, sizeof(p.rk0));
    std::memcpy(p.rk1, ctx->rk1, sizeof(p.rk1));
    return p;
}

// Kernel-node parameters of the chunk graph for one chunk [t0, t0 + n).
// `pp` / `rp` hold one StepParams per node (kernelParams point into them).
void chunk_params(const bd_ctx* ctx, int64_t t0, int64_t n, std::vector<StepParams>& pp,
                  std::vector<StepParams>& rp)
{
    StepParams p = base_params(ctx);
    p.t0 = t0; p.n_steps = n;
    pp.assign(ctx->par_classes.size(), p);
    for (size_t k = 0; k < ctx->par_classes.size(); ++k) {
        const ParClass& pc = ctx->par_classes[k];
        pp[k].parent_warps = ctx->d_parent_warps + pc.warp_begin;
        pp[k].n_parent_warps = pc.warp_count;
    }
    rp.assign(ctx->var_classes.size(), p);
    for (size_t k = 0; k < ctx->var_classes.size(); ++k) {
        const VarClass& vc = ctx->var_classes[k];
        rp[k].items = ctx->d_items + vc.item_begin;
        rp[k].n_items = vc.item_count;
        rp[k].queue = ctx->d_queue + k;
    }
}

cudaKernelNodeParams parent_node(const bd_ctx* ctx, size_t k, StepParams* pk, void** args)
{
    const ParClass& pc = ctx->par_classes[k];
    args[0] = pk;
    cudaKernelNodeParams kp = {};
    if (pc.hi)
        kp.func = const_cast<void*>(ctx->f64 ? hi_parent_func_f64(pc.L == 0) : hi_parent_func_f32(pc.L == 0));
    else
        kp.func = const_cast<void*>(ctx->f64 ? parent_func_f64(pc.L, pc.lj) : parent_func_f32(pc.L, pc.lj));
    kp.gridDim = dim3(pc.grid);
    kp.blockDim = dim3(pc.threads);
    kp.sharedMemBytes = (unsigned)pc.smem;
    kp.kernelParams = args;
    return kp;
}

cudaKernelNodeParams replica_node(const bd_ctx* ctx, size_t k, StepParams* rk, void** args)
{
    const VarClass& vc = ctx->var_classes[k];
    args[0] = rk;
    cudaKernelNodeParams kp = {};
    if (variant_hi(vc.variant))
        kp.func = const_cast<void*>(ctx->f64 ? hi_replica_func_f64(vc.variant == kHIBase)
                                             : hi_replica_func_f32(vc.variant == kHIBase));
    else
        kp.func = const_cast<void*>(ctx->f64 ? persist_func_f64(vc.variant, ctx->conf)
                                             : persist_func_f32(vc.variant, ctx->conf));
    kp.gridDim = dim3(vc.grid);
    kp.blockDim = dim3(vc.threads);
    kp.sharedMemBytes = (unsigned)vc.smem;
    kp.kernelParams = args;
    return kp;
}

// Kernel-node parameters of the fold of windows [w0, w1) (grid of at least one block).
cudaKernelNodeParams fold_node_params(const bd_ctx* ctx, int64_t w0, int64_t w1, FoldParams* fp,
                                      void** args)
{
    fp->chains = ctx->d_chains;
    fp->spring_chain = ctx->d_spring_chain;
    fp->part = ctx->d_part;
    fp->rsf = ctx->d_rsf;
    fp->M = ctx->M;
    fp->part_stride = ctx->part_stride;
    fp->w0 = w0;
    fp->w1 = w1;
    fp->ring = ctx->part_ring;
    fp->pad = 0;
    fp->bead_chain = ctx->d_bead_chain;
    fp->dpart = ctx->d_dpart;
    fp->dbead = ctx->d_dbead;
    fp->NB = ctx->conf ? ctx->n_beads : 0;
    fp->bpart_stride = ctx->bpart_stride;
    args[0] = fp;
    const int th = rsf_fold_threads();
    const int64_t n = std::max<int64_t>(1, (w1 - w0) * (ctx->M + fp->NB));
    cudaKernelNodeParams kp = {};
    kp.func = const_cast<void*>(rsf_fold_func());
    kp.gridDim = dim3((unsigned)((n + th - 1) / th));
    kp.blockDim = dim3(th);
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    return kp;
}

void drop_graph(bd_ctx* ctx)
{
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    if (ctx->graph) cudaGraphDestroy(ctx->graph);
    ctx->gexec = nullptr;
    ctx->graph = nullptr;
    ctx->par_nodes.clear();
    ctx->rep_nodes.clear();
    cudaGetLastError();
}

// Builds the chunk graph: start event -> queue reset -> parent kernels (one
// per tile, parallel) -> mid event -> replica kernels (one per variant,
// parallel) -> end event.
bd_status build_graph(bd_ctx* ctx)
{
    drop_graph(ctx);
    for (int i = 0; i < 3; ++i)
        if (!ctx->idle_ev[i]) BD_CUDA(ctx, cudaEventCreate(&ctx->idle_ev[i]));
    BD_CUDA(ctx, cudaGraphCreate(&ctx->graph, 0));
    std::vector<StepParams> pp, rp;
    chunk_params(ctx, 0, 0, pp, rp);
    cudaGraphNode_t prev;
    BD_CUDA(ctx, cudaGraphAddEventRecordNode(&ctx->ev_nodes[0], ctx->graph, nullptr, 0, ctx->idle_ev[0]));
    cudaMemsetParams ms = {};
    ms.dst = ctx->d_queue;
    ms.value = 0;
    ms.elementSize = sizeof(int32_t);
    ms.width = ctx->var_classes.size();
    ms.height = 1;
    ms.pitch = 0;
    cudaGraphNode_t mnode;
    BD_CUDA(ctx, cudaGraphAddMemsetNode(&mnode, ctx->graph, &ctx->ev_nodes[0], 1, &ms));
    prev = mnode;
    for (size_t k = 0; k < ctx->par_classes.size(); ++k) {      // parallel branches
        void* args[1];
        cudaKernelNodeParams kp = parent_node(ctx, k, &pp[k], args);
        cudaGraphNode_t nd;
        BD_CUDA(ctx, cudaGraphAddKernelNode(&nd, ctx->graph, &prev, 1, &kp));
        ctx->par_nodes.push_back(nd);
    }
    BD_CUDA(ctx, cudaGraphAddEventRecordNode(&ctx->ev_nodes[1], ctx->graph, ctx->par_nodes.data(),
                                             ctx->par_nodes.size(), ctx->idle_ev[1]));
    for (size_t k = 0; k < ctx->var_classes.size(); ++k) {
        void* args[1];
        cudaKernelNodeParams kp = replica_node(ctx, k, &rp[k], args);
        cudaGraphNode_t nd;
        BD_CUDA(ctx, cudaGraphAddKernelNode(&nd, ctx->graph, &ctx->ev_nodes[1], 1, &kp));
        ctx->rep_nodes.push_back(nd);
    }
    BD_CUDA(ctx, cudaGraphAddEventRecordNode(&ctx->ev_nodes[2], ctx->graph, ctx->rep_nodes.data(),
                                             ctx->rep_nodes.size(), ctx->idle_ev[2]));
    {
        FoldParams fp;
        void* args[1];
        cudaKernelNodeParams kp = fold_node_params(ctx, 0, 0, &fp, args);
        BD_CUDA(ctx, cudaGraphAddKernelNode(&ctx->fold_node, ctx->graph, &ctx->ev_nodes[2], 1, &kp));
    }
    BD_CUDA(ctx, cudaGraphInstantiate(&ctx->gexec, ctx->graph, 0));
    return BD_OK;
}

bd_status reset_kinetics(bd_ctx* ctx)
{
    const int64_t M = ctx->M;
    BD_CUDA(ctx, cudaMemsetAsync(ctx->d_lam, 0, sizeof(double) * 3 * M, ctx->stream));
    BD_CUDA(ctx, cudaMemsetAsync(ctx->d_first_thr, 0xff, sizeof(int64_t) * 3 * M, ctx->stream));
    BD_CUDA(ctx, cudaMemsetAsync(ctx->d_first_bell, 0xff, sizeof(int64_t) * 3 * M, ctx->stream));
    BD_CUDA(ctx, cudaMemsetAsync(ctx->d_tsf_acc, 0, sizeof(double) * M, ctx->stream));
    BD_CUDA(ctx, cudaMemsetAsync(ctx->d_overext, 0, sizeof(unsigned long long) * ctx->cfg.n_chains,
                                 ctx->stream));
    return BD_OK;
}

bd_status load_positions(bd_ctx* ctx, const double* pos)
{
    const size_t n = sizeof(double) * 3 * (size_t)ctx->n_beads;
    const double* src = pos;
    if (!is_device_ptr(pos)) {
        bd_status s = ensure_io(ctx, n);
        if (s != BD_OK) return s;
        BD_CUDA(ctx, cudaMemcpyAsync(ctx->d_io, pos, n, cudaMemcpyHostToDevice, ctx->stream));
        src = (const double*)ctx->d_io;
    }
    ++ctx->launches;
    BD_CUDA(ctx, run_set_bonds(ctx->f64, ctx->d_chains, ctx->d_spring_chain, ctx->M, src,
                               ctx->d_state, ctx->stream));
    if (src != pos) BD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return BD_OK;
}

// Applies the TSF / RSF criteria to windows completed since the last call.
bd_status apply_windows(bd_ctx* ctx)
{
    const int64_t done = ctx->step / ctx->cfg.window_steps;
    if (done > ctx->windows_detected) {
        ++ctx->launches;
        BD_CUDA(ctx, run_window_criteria(ctx->d_chains, ctx->d_spring_chain, ctx->M, ctx->d_rsf,
                                         ctx->d_tsf, ctx->windows_detected, done,
                                         ctx->cfg.window_steps, ctx->cfg.dt, ctx->cfg.thr_mask,
                                         ctx->cfg.bell_mask, ctx->d_exp1, ctx->d_lam,
                                         ctx->d_first_thr, ctx->d_first_bell, ctx->stream));
        ctx->windows_detected = done;
    }
    return BD_OK;
}

// Writes n bytes produced on the device at `dev` to out (host or device).
bd_status deliver(bd_ctx* ctx, void* out, const void* dev, size_t n, bool out_is_dev)
{
    if (out_is_dev) {
        if (out != dev) BD_CUDA(ctx, cudaMemcpyAsync(out, dev, n, cudaMemcpyDeviceToDevice, ctx->stream));
        return BD_OK;
    }
    BD_CUDA(ctx, cudaMemcpyAsync(out, dev, n, cudaMemcpyDeviceToHost, ctx->stream));
    BD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return BD_OK;
}

template <typename T>
bd_status upload(bd_ctx* ctx, T** dst, const std::vector<T>& v)
{
    bd_status s = dalloc(ctx, (void**)dst, sizeof(T) * std::max<size_t>(v.size(), 1));
    if (s != BD_OK) return s;
    if (!v.empty())
        BD_CUDA(ctx, cudaMemcpyAsync(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice,
                                     ctx->stream));
    return BD_OK;
}

void release(bd_ctx* ctx)
{
    if (!ctx) return;
    if (!ctx->allocs.empty()) cudaStreamSynchronize(ctx->stream);
    drop_graph(ctx);
    for (int i = 0; i < 3; ++i)
        if (ctx->idle_ev[i]) { cudaEventDestroy(ctx->idle_ev[i]); ctx->idle_ev[i] = nullptr; }
    cudaEvent_t* evs[] = {&ctx->ev_init, &ctx->ev_done, &ctx->ev_win[0], &ctx->ev_win[1],
                          &ctx->ev_mu_free[0], &ctx->ev_mu_free[1], &ctx->ev_seg_free[0],
                          &ctx->ev_seg_free[1]};
    for (cudaEvent_t* e : evs)
        if (*e) { cudaEventDestroy(*e); *e = nullptr; }
    if (ctx->adj_stream) { cudaStreamDestroy(ctx->adj_stream); ctx->adj_stream = nullptr; }
    for (void* p : ctx->allocs) cudaFree(p);
    ctx->allocs.clear();
    cudaGetLastError();
}

// Measured issue cost per warp-step of each variant, per (device,
// precision), shared by every context of the process.
std::mutex g_tune_mutex;
std::map<std::pair<int, int>, std::vector<double>> g_tune_cache;

// Times every compiled step variant on the context's own chains: a scratch
// copy of the state, steps 1 .. probe_steps of a window too long to end (no
// spawn, no window-end reduction), enough warp items to fill the GPU four
// times over. cost[v] = kernel time / (work items x steps): the GPU's
// throughput cost of one warp-step of variant v, in nanoseconds.
bd_status autotune_probe(bd_ctx* ctx, int probe_steps, std::vector<double>& cost)
{
    cost.assign(kVariantCodes, 0.0);
    const int* vars = ctx->f64 ? kVariantsF64 : kVariantsF32;
    const int nv = ctx->f64 ? kNumVariantsF64 : kNumVariantsF32;
    const int threads = ctx->f64 ? persist_threads_f64() : persist_threads_f32();
    const size_t state_bytes = ctx->tsize * 3 * (size_t)ctx->state_bonds;
    void* tstate = nullptr;
    unsigned long long* tover = nullptr;
    int32_t* tqueue = nullptr;
    ItemDev* titems = nullptr;
    size_t titems_cap = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    bd_status st = BD_OK;
#define BD_PROBE(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) { cudaGetLastError(); st = fail(ctx, BD_E_CUDA, "autotune: %s failed: %s", #call, cudaGetErrorString(e_)); goto done; } } while (0)
    BD_PROBE(cudaMalloc(&tstate, state_bytes));
    BD_PROBE(cudaMalloc((void**)&tover, sizeof(unsigned long long) * ctx->cfg.n_chains));
    BD_PROBE(cudaMalloc((void**)&tqueue, sizeof(int32_t)));
    BD_PROBE(cudaMemcpyAsync(tstate, ctx->d_state, state_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    BD_PROBE(cudaEventCreate(&e0));
    BD_PROBE(cudaEventCreate(&e1));
    for (int t = 0; t < nv; ++t) {
        const int v = vars[t];
        const int L = variant_tile(v);
        std::vector<ItemDev> items;
        for (int c = 0; c < ctx->cfg.n_chains; ++c) {
            const int N = ctx->chains[c].n_beads, R = ctx->chains[c].n_replicas;
            const int G = (N + L - 1) / L;
            const bool rest_law = ctx->chains[c].spring == BD_SPRING_HARMONIC || ctx->chains[c].spring == BD_SPRING_VWF;
            if (G > 32 || variant_lj(v) != rest_law ||
                ctx->chains[c].hi_a > 0) continue;
            const int per_warp = (variant_paired(v) ? 2 : 1) * (32 / G);
            split_replicas(c, R, per_warp, v, items);
        }
        if (items.empty()) continue;
        int per_sm = 1;
        BD_PROBE(ctx->f64 ? persist_blocks_per_sm_f64(v, false, &per_sm) : persist_blocks_per_sm_f32(v, false, &per_sm));
        const size_t resident = (size_t)per_sm * ctx->n_sm * (threads / 32);
        const size_t base = items.size();
        while (items.size() < 4 * resident) items.push_back(items[items.size() % base]);
        order_items(items);
        if (items.size() > titems_cap) {
            if (titems) cudaFree(titems);
            titems = nullptr;
            BD_PROBE(cudaMalloc((void**)&titems, sizeof(ItemDev) * items.size()));
            titems_cap = items.size();
        }
        BD_PROBE(cudaMemcpyAsync(titems, items.data(), sizeof(ItemDev) * items.size(),
                                 cudaMemcpyHostToDevice, ctx->stream));
        StepParams p = base_params(ctx);
        p.state = tstate;
        p.overext = tover;
        p.items = titems;
        p.n_items = (int32_t)items.size();
        p.queue = tqueue;
        p.S = 1 << 30;                 // no window starts or ends inside the probe
        p.t0 = 1;
        p.n_steps = probe_steps;
        void* args[1] = {&p};
        const void* fn = ctx->f64 ? persist_func_f64(v, false) : persist_func_f32(v, false);
        const dim3 grid((unsigned)std::max<size_t>(1, std::min<size_t>((items.size() + threads / 32 - 1) / (threads / 32), (size_t)per_sm * ctx->n_sm)));
        for (int rep = 0; rep < 2; ++rep) {      // first launch warms up
            BD_PROBE(cudaMemsetAsync(tqueue, 0, sizeof(int32_t), ctx->stream));
            BD_PROBE(cudaEventRecord(e0, ctx->stream));
            BD_PROBE(cudaLaunchKernel(fn, grid, dim3(threads), args,
                                      ctx->f64 ? persist_smem_f64(v) : persist_smem_f32(v), ctx->stream));
            BD_PROBE(cudaEventRecord(e1, ctx->stream));
            ++ctx->launches;
        }
        BD_PROBE(cudaEventSynchronize(e1));
        float ms = 0.0f;
        BD_PROBE(cudaEventElapsedTime(&ms, e0, e1));
        cost[v] = (double)ms * 1e6 / ((double)items.size() * probe_steps);
    }
done:
#undef BD_PROBE
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(ctx->stream);
    if (titems) cudaFree(titems);
    if (tqueue) cudaFree(tqueue);
    if (tover) cudaFree(tover);
    if (tstate) cudaFree(tstate);
    cudaGetLastError();
    return st;
}

// Re-plans with the current variant costs and rebuilds what depends on the
// plan (chain table, work items, partial-sum history, queues, graph). Only
// valid before the first window completes.
bd_status replan(bd_ctx* ctx)
{
    BD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const size_t old_items = ctx->h_items.size();
    const int64_t old_part = ctx->part_stride;
    const int64_t old_bpart = ctx->bpart_stride;
    const size_t old_queue = ctx->var_classes.size();
    bd_status s = plan(ctx);
    if (s != BD_OK) return s;
    BD_CUDA(ctx, cudaMemcpyAsync(ctx->d_chains, ctx->h_chains.data(), sizeof(ChainDev) * ctx->h_chains.size(),
                                 cudaMemcpyHostToDevice, ctx->stream));
    dfree(ctx, ctx->d_items, sizeof(ItemDev) * std::max<size_t>(old_items, 1));
    ctx->d_items = nullptr;
    if ((s = upload(ctx, &ctx->d_items, ctx->h_items)) != BD_OK) return s;
    dfree(ctx, ctx->d_part, std::max<size_t>(sizeof(double) * (size_t)ctx->part_ring * (size_t)old_part, 16));
    ctx->d_part = nullptr;
    if ((s = dalloc(ctx, (void**)&ctx->d_part, sizeof(double) * (size_t)ctx->part_ring * (size_t)ctx->part_stride)) != BD_OK)
        return s;
    if (ctx->conf) {
        dfree(ctx, ctx->d_dpart, std::max<size_t>(sizeof(double) * 3 * (size_t)ctx->part_ring * (size_t)old_bpart, 16));
        ctx->d_dpart = nullptr;
        if ((s = dalloc(ctx, (void**)&ctx->d_dpart, sizeof(double) * 3 * (size_t)ctx->part_ring *
                                                        (size_t)ctx->bpart_stride)) != BD_OK)
            return s;
    }
    dfree(ctx, ctx->d_queue, std::max<size_t>(sizeof(int32_t) * old_queue, 16));
    ctx->d_queue = nullptr;
    if ((s = dalloc(ctx, (void**)&ctx->d_queue, sizeof(int32_t) * ctx->var_classes.size())) != BD_OK) return s;
    return build_graph(ctx);
}


// ---------------------------------------------------------------------------
// Adjoint plan: per chain the smallest replica tile of kAdjTiles that fits a
// replica in one warp, its replicas split into warp items of up to 32 / G;
// checkpoint storage for every K steps of max_windows windows.
// ---------------------------------------------------------------------------
bd_status adj_plan(bd_ctx* ctx)
{
    const bd_config& cfg = ctx->cfg;
    const int C = cfg.n_chains;
    ctx->h_adj.assign(C, AdjChain{});
    std::vector<std::pair<int, ItemDev>> items;
    int64_t part = 0;
    for (int c = 0; c < C; ++c) {
        const bd_chain_desc& d = ctx->chains[c];
        int L = 0;
        for (int t = 0; t < kNumAdjTiles && !L; ++t)
            if ((d.n_beads + kAdjTiles[t] - 1) / kAdjTiles[t] <= 32) L = kAdjTiles[t];
        if (!L) return fail(ctx, BD_E_INVALID, "chain %d: no adjoint tile fits N=%d", c, d.n_beads);
        const int G = (d.n_beads + L - 1) / L, P = 32 / G;
        const int groups = (d.n_replicas + P - 1) / P;
        AdjChain& a = ctx->h_adj[c];
        a.part_off = part;
        a.n_groups = groups;
        a.pad = 0;
        a.khat[0] = a.khat[1] = a.khat[2] = a.khat[3] = 0.0;
        switch (d.flow) {
        case BD_FLOW_SHEAR: a.khat[3] = 1.0; break;
        case BD_FLOW_UNIAXIAL: a.khat[0] = 1.0; a.khat[1] = -0.5; a.khat[2] = -0.5; break;
        case BD_FLOW_PLANAR: a.khat[0] = 1.0; a.khat[1] = -1.0; break;
        default: break;
        }
        int begin = 0;
        for (int g = 0; g < groups; ++g) {
            const int cnt = d.n_replicas / groups + (g < d.n_replicas % groups ? 1 : 0);
            items.push_back({L, ItemDev{c, g, begin, cnt, L, 1}});
            begin += cnt;
        }
        part += (int64_t)groups * (d.n_beads - 1);
    }
    ctx->adj_stride = part;
    std::stable_sort(items.begin(), items.end(),
                     [](const std::pair<int, ItemDev>& x, const std::pair<int, ItemDev>& y) { return x.first < y.first; });
    ctx->h_adj_items.clear();
    ctx->adj_classes.clear();
    for (size_t k = 0; k < items.size(); ++k) {
        if (ctx->adj_classes.empty() || ctx->adj_classes.back().L != items[k].first)
            ctx->adj_classes.push_back(AdjClass{items[k].first, (int)k, 0});
        ctx->adj_classes.back().item_count++;
        ctx->h_adj_items.push_back(items[k].second);
    }
    bd_status s;
    if ((s = upload(ctx, &ctx->d_adj, ctx->h_adj)) != BD_OK) return s;
    if ((s = upload(ctx, &ctx->d_adj_items, ctx->h_adj_items)) != BD_OK) return s;
    ctx->n_ckpt = cfg.max_windows * (int64_t)cfg.window_steps / cfg.checkpoint_steps + 1;
    return dalloc(ctx, &ctx->d_ckpt, ctx->tsize * 3 * (size_t)ctx->M * (size_t)ctx->n_ckpt);
}

// Work buffers of bd_adjoint: a K-row parent segment, the parent adjoint,
// and replica-window batches sized to a quarter of the free device memory
// (between 1 and 32 GiB).
bd_status adj_buffers(bd_ctx* ctx)
{
    if (ctx->d_seg[0]) return BD_OK;
    const int64_t K = ctx->cfg.checkpoint_steps, S = ctx->cfg.window_steps, M = ctx->M;
    const size_t per_window = ctx->tsize * 3 * (size_t)ctx->state_bonds * (size_t)(S + 1) +
                              sizeof(double) * 3 * 2 * (size_t)ctx->adj_stride;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        free_b = 0;
    }
    const int64_t budget = std::min<int64_t>(32ll << 30, std::max<int64_t>(1ll << 30, (int64_t)(free_b / 4)));
    ctx->rep_batch = std::max<int64_t>(1, std::min<int64_t>({K / S, 65535, budget / (int64_t)per_window}));
    BD_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->adj_stream, cudaStreamNonBlocking));
    cudaEvent_t* evs[] = {&ctx->ev_init, &ctx->ev_done, &ctx->ev_win[0], &ctx->ev_win[1],
                          &ctx->ev_mu_free[0], &ctx->ev_mu_free[1], &ctx->ev_seg_free[0],
                          &ctx->ev_seg_free[1]};
    for (cudaEvent_t* e : evs) BD_CUDA(ctx, cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    bd_status s;
    for (int b = 0; b < 2; ++b) {
        if ((s = dalloc(ctx, &ctx->d_seg[b], ctx->tsize * 3 * (size_t)M * (size_t)K)) != BD_OK) return s;
        if ((s = dalloc(ctx, (void**)&ctx->d_mu[b], sizeof(double) * 3 * (size_t)ctx->adj_stride *
                                                        (size_t)ctx->rep_batch)) != BD_OK) return s;
    }
    if ((s = dalloc(ctx, &ctx->d_lamP, ctx->tsize * 3 * (size_t)M)) != BD_OK) return s;
    if ((s = dalloc(ctx, &ctx->d_repbuf, ctx->tsize * 3 * (size_t)ctx->state_bonds * (size_t)(S + 1) *
                                             (size_t)ctx->rep_batch)) != BD_OK) return s;
    if ((s = dalloc(ctx, (void**)&ctx->d_gls, sizeof(double) * (size_t)ctx->cfg.n_chains)) != BD_OK) return s;
    return dalloc(ctx, (void**)&ctx->d_grad, sizeof(double) * 3 * (size_t)ctx->cfg.n_chains);
}

// Keeps the parent checkpoints of the windows [w_first, w_end) whose
// snapshots the last chunk wrote (rows w - w_first of the snapshot buffer).
bd_status keep_checkpoints(bd_ctx* ctx, int64_t w_first, int64_t w_end)
{
    const int64_t K = ctx->cfg.checkpoint_steps, S = ctx->cfg.window_steps;
    const size_t row = ctx->tsize * 3 * (size_t)ctx->M;
    for (int64_t w = w_first; w < w_end; ++w) {
        const int64_t t = w * S - ctx->origin;
        if (t < 0 || t % K) continue;
        const int64_t j = t / K;
        if (j >= ctx->n_ckpt) continue;
        BD_CUDA(ctx, cudaMemcpyAsync((char*)ctx->d_ckpt + j * row, (const char*)ctx->d_snap + (w % ctx->part_ring) * row,
                                     row, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    return BD_OK;
}

bd_status adj_launch(bd_ctx* ctx, int kind, int L, dim3 grid, AdjParams* a, cudaStream_t st)
{
    const void* fn = ctx->f64 ? adj_func_f64(kind, L) : adj_func_f32(kind, L);
    if (!fn) return fail(ctx, BD_E_INVALID, "no adjoint kernel %d for tile %d", kind, L);
    void* args[1] = {a};
    BD_CUDA(ctx, cudaLaunchKernel(fn, grid, dim3(kAdjThreads), args, 0, st));
    ++ctx->launches;
    return BD_OK;
}

// Parent kernels of the adjoint over every parent tile.
bd_status adj_parents(bd_ctx* ctx, int kind, AdjParams a, cudaStream_t st)
{
    for (const ParClass& pc : ctx->par_classes) {
        a.sp.parent_warps = ctx->d_parent_warps + pc.warp_begin;
        a.sp.n_parent_warps = pc.warp_count;
        const int per_cta = kAdjThreads / 32;
        bd_status s = adj_launch(ctx, kind, pc.L, dim3((pc.warp_count + per_cta - 1) / per_cta), &a, st);
        if (s != BD_OK) return s;
    }
    return BD_OK;
}
// Kernels whose bounded waits gave up leave bits in the context's device
// error word (StepParams::dev_err); the calls below that synchronise the
// stream report them as BD_E_TIMEOUT.
bd_status check_device_error(bd_ctx* ctx)
{
    int32_t e = 0;
    BD_CUDA(ctx, cudaMemcpyAsync(&e, ctx->d_dev_err, sizeof(e), cudaMemcpyDeviceToHost, ctx->stream));
    BD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (e)
        return fail(ctx, BD_E_TIMEOUT, "a tensor-core completion wait gave up (device error bits 0x%x); "
                    "the steps run since are not valid", (unsigned)e);
    return BD_OK;
}

}  // namespace

extern "C" {

const char* bd_status_string(bd_status s)
{
    switch (s) {
    case BD_OK: return "BD_OK";
    case BD_E_INVALID: return "BD_E_INVALID";
    case BD_E_CUDA: return "BD_E_CUDA";
    case BD_E_OOM: return "BD_E_OOM";
    case BD_E_STATE: return "BD_E_STATE";
    case BD_E_TIMEOUT: return "BD_E_TIMEOUT";
    case BD_E_CAPACITY: return "BD_E_CAPACITY";
    }
    return "BD_E_UNKNOWN";
}

const char* bd_last_error(const bd_ctx* ctx)
{
    if (!ctx) return "NULL context";
    return ctx->err.c_str();
}

bd_status bd_create(const bd_config* cfg, const double* init_pos, bd_ctx** out)
{
    if (!out) return BD_E_INVALID;
    *out = nullptr;
    bd_ctx* ctx = new (std::nothrow) bd_ctx();
    if (!ctx) return BD_E_OOM;
    bd_status s = validate(ctx, cfg);
    if (s == BD_OK && !init_pos) s = fail(ctx, BD_E_INVALID, "init_pos is NULL");
    if (s != BD_OK) { delete ctx; return s; }
    ctx->cfg = *cfg;
    ctx->chains.assign(cfg->chains, cfg->chains + cfg->n_chains);
    ctx->cfg.chains = ctx->chains.data();
    ctx->stream = (cudaStream_t)cfg->stream;
    ctx->f64 = cfg->precision == BD_PREC_FP64;
    ctx->conf = (cfg->flags & BD_FLAG_CONFORMATION) != 0;
    ctx->tsize = ctx->f64 ? sizeof(double) : sizeof(float);
    round_keys(cfg->seed, ctx->rk0, ctx->rk1);

#define BD_TRY(x) do { s = (x); if (s != BD_OK) goto failed; } while (0)
    {
        cudaError_t e = cudaGetDevice(&ctx->device);
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, ctx->device);
        if (e != cudaSuccess) { cudaGetLastError(); s = fail(ctx, BD_E_CUDA, "no CUDA device: %s", cudaGetErrorString(e)); goto failed; }
    }
    for (int v = 0; v < kVariantCodes; ++v) ctx->var_cost[v] = default_variant_cost(v);
    BD_TRY(plan(ctx));
    {
        const int64_t M = ctx->M, C = cfg->n_chains, W = cfg->max_windows;
        std::vector<int32_t> spring_chain(M);
        std::vector<int64_t> pair_parent(C + 1), pair_all(C + 1);
        pair_parent[0] = pair_all[0] = 0;
        for (int c = 0; c < C; ++c) {
            for (int i = 0; i < ctx->chains[c].n_beads - 1; ++i)
                spring_chain[ctx->h_chains[c].spr_off + i] = c;
            pair_parent[c + 1] = pair_parent[c] + 1;
            pair_all[c + 1] = pair_all[c] + ctx->chains[c].n_replicas + 1;
        }
        BD_TRY(upload(ctx, &ctx->d_chains, ctx->h_chains));
        BD_TRY(upload(ctx, &ctx->d_items, ctx->h_items));
        BD_TRY(upload(ctx, &ctx->d_parent_items, ctx->h_parent_items));
        BD_TRY(upload(ctx, &ctx->d_parent_warps, ctx->h_parent_warps));
        BD_TRY(upload(ctx, &ctx->d_spring_chain, spring_chain));
        BD_TRY(upload(ctx, &ctx->d_pair_parent, pair_parent));
        BD_TRY(upload(ctx, &ctx->d_pair_all, pair_all));
        BD_TRY(dalloc(ctx, &ctx->d_state, ctx->tsize * 3 * (size_t)ctx->state_bonds));
        BD_TRY(dalloc(ctx, &ctx->d_snap, ctx->tsize * 3 * (size_t)M * (size_t)(ctx->chunk_windows + 1)));
        ctx->part_ring = (int32_t)(ctx->chunk_windows + 1);
        BD_TRY(dalloc(ctx, (void**)&ctx->d_part, sizeof(double) * (size_t)ctx->part_ring * (size_t)ctx->part_stride));
        BD_TRY(dalloc(ctx, (void**)&ctx->d_rsf, sizeof(double) * (size_t)W * (size_t)M));
        if (ctx->conf) {
            std::vector<int32_t> bead_chain(ctx->n_beads);
            for (int c = 0; c < C; ++c)
                for (int i = 0; i < ctx->chains[c].n_beads; ++i) bead_chain[ctx->h_chains[c].bead_off + i] = c;
            BD_TRY(upload(ctx, &ctx->d_bead_chain, bead_chain));
            BD_TRY(dalloc(ctx, (void**)&ctx->d_dbar, sizeof(double) * 3 * (size_t)W * (size_t)ctx->n_rep));
            BD_TRY(dalloc(ctx, (void**)&ctx->d_dpart, sizeof(double) * 3 * (size_t)ctx->part_ring *
                                                          (size_t)ctx->bpart_stride));
            BD_TRY(dalloc(ctx, (void**)&ctx->d_dbead, sizeof(double) * 3 * (size_t)W * (size_t)ctx->n_beads));
            BD_TRY(dalloc(ctx, (void**)&ctx->d_rgz, sizeof(double) * (size_t)W * (size_t)C));
        }
        BD_TRY(dalloc(ctx, (void**)&ctx->d_tsf, sizeof(double) * (size_t)W * (size_t)M));
        BD_TRY(dalloc(ctx, (void**)&ctx->d_tsf_acc, sizeof(double) * (size_t)M));
        BD_TRY(dalloc(ctx, (void**)&ctx->d_lam, sizeof(double) * 3 * (size_t)M));
        BD_TRY(dalloc(ctx, (void**)&ctx->d_first_thr, sizeof(int64_t) * 3 * (size_t)M));
        BD_TRY(dalloc(ctx, (void**)&ctx->d_first_bell, sizeof(int64_t) * 3 * (size_t)M));
        BD_TRY(dalloc(ctx, (void**)&ctx->d_exp1, sizeof(double) * 3 * (size_t)M));
        BD_TRY(dalloc(ctx, (void**)&ctx->d_overext, sizeof(unsigned long long) * (size_t)C));
        BD_TRY(dalloc(ctx, (void**)&ctx->d_dev_err, sizeof(int32_t)));
        if (cudaMemsetAsync(ctx->d_dev_err, 0, sizeof(int32_t), ctx->stream) != cudaSuccess) {
            cudaGetLastError();
            s = fail(ctx, BD_E_CUDA, "device error word");
            goto failed;
        }
        BD_TRY(dalloc(ctx, (void**)&ctx->d_evt_scratch, sizeof(int64_t) * (size_t)(event_blocks(M) + 1)));
        BD_TRY(dalloc(ctx, (void**)&ctx->d_queue, sizeof(int32_t) * ctx->var_classes.size()));
        BD_TRY(build_graph(ctx));
        if (cfg->checkpoint_steps > 0) BD_TRY(adj_plan(ctx));
        {
            cudaError_t e = run_exp1(ctx->d_chains, ctx->d_spring_chain, M, ctx->rk0[0], ctx->rk1[0],
                                     (uint32_t)cfg->chain_id_base, ctx->d_exp1, ctx->stream);
            if (e != cudaSuccess) { cudaGetLastError(); s = fail(ctx, BD_E_CUDA, "exp1: %s", cudaGetErrorString(e)); goto failed; }
        }
        BD_TRY(reset_kinetics(ctx));
        BD_TRY(load_positions(ctx, init_pos));
        {
            cudaError_t e = cudaStreamSynchronize(ctx->stream);
            if (e != cudaSuccess) { cudaGetLastError(); s = fail(ctx, BD_E_CUDA, "set-up: %s", cudaGetErrorString(e)); goto failed; }
        }
    }
#undef BD_TRY
    *out = ctx;
    return BD_OK;
failed:
    release(ctx);
    delete ctx;
    return s;
}

void bd_destroy(bd_ctx* ctx)
{
    if (!ctx) return;
    release(ctx);
    delete ctx;
}

bd_status bd_spawn_replicas(bd_ctx* ctx)
{
    if (!ctx) return BD_E_INVALID;
    ++ctx->launches;
    BD_CUDA(ctx, run_spawn(ctx->f64, ctx->d_chains, ctx->d_spring_chain, ctx->M, ctx->d_state,
                           ctx->stream));
    return BD_OK;
}

bd_status bd_step(bd_ctx* ctx, int64_t n_steps)
{
    if (!ctx) return BD_E_INVALID;
    if (n_steps < 0) return fail(ctx, BD_E_INVALID, "n_steps must be >= 0");
    if (n_steps == 0) return BD_OK;
    const int64_t S = ctx->cfg.window_steps;
    const int64_t t_end = ctx->step + n_steps;
    if (t_end > (int64_t)UINT32_MAX)
        return fail(ctx, BD_E_CAPACITY, "step counter would pass 2^32 (noise counter word)");
    if (t_end / S > ctx->cfg.max_windows)
        return fail(ctx, BD_E_CAPACITY, "run to step %lld needs %lld windows; max_windows is %lld",
                    (long long)t_end, (long long)(t_end / S), (long long)ctx->cfg.max_windows);
    std::vector<StepParams> pp, rp;
    std::vector<void*> pargs(ctx->par_nodes.size()), rargs(ctx->rep_nodes.size());
    int64_t t = ctx->step;
    while (t < t_end) {
        const int64_t w_first = (t + S - 1) / S;
        const int64_t chunk_end = std::min(t_end, (w_first + ctx->chunk_windows) * S);
        chunk_params(ctx, t, chunk_end - t, pp, rp);
        for (size_t k = 0; k < ctx->par_nodes.size(); ++k) {
            cudaKernelNodeParams kp = parent_node(ctx, k, &pp[k], &pargs[k]);
            BD_CUDA(ctx, cudaGraphExecKernelNodeSetParams(ctx->gexec, ctx->par_nodes[k], &kp));
        }
        for (size_t k = 0; k < ctx->rep_nodes.size(); ++k) {
            cudaKernelNodeParams kp = replica_node(ctx, k, &rp[k], &rargs[k]);
            BD_CUDA(ctx, cudaGraphExecKernelNodeSetParams(ctx->gexec, ctx->rep_nodes[k], &kp));
        }
        {   // fold the windows this chunk completes, [t / S, chunk_end / S), into the RSF history
            FoldParams fp;
            void* fargs[1];
            cudaKernelNodeParams kp = fold_node_params(ctx, t / S, chunk_end / S, &fp, fargs);
            BD_CUDA(ctx, cudaGraphExecKernelNodeSetParams(ctx->gexec, ctx->fold_node, &kp));
        }
        BD_CUDA(ctx, cudaGraphLaunch(ctx->gexec, ctx->stream));
        ctx->launches += (int64_t)(ctx->par_nodes.size() + ctx->rep_nodes.size() + 1);
        if (ctx->cfg.checkpoint_steps > 0) {
            bd_status s = keep_checkpoints(ctx, w_first, (chunk_end + S - 1) / S);
            if (s != BD_OK) return s;
        }
        if (ctx->timing) {
            // the graph's own events: read them before the next launch re-records them
            float x = 0.0f, y = 0.0f;
            BD_CUDA(ctx, cudaEventSynchronize(ctx->idle_ev[2]));
            BD_CUDA(ctx, cudaEventElapsedTime(&x, ctx->idle_ev[0], ctx->idle_ev[1]));
            BD_CUDA(ctx, cudaEventElapsedTime(&y, ctx->idle_ev[1], ctx->idle_ev[2]));
            ctx->timed_ms[0] += x;
            ctx->timed_ms[1] += y;
            ctx->timed_n[0] += (int64_t)ctx->par_nodes.size();
            ctx->timed_n[1] += (int64_t)ctx->rep_nodes.size();
        }
        t = chunk_end;
        ctx->step = t;
    }
    return BD_OK;
}

bd_status bd_replica_average(bd_ctx* ctx, int64_t window, double* out)
{
    if (!ctx || !out) return ctx ? fail(ctx, BD_E_INVALID, "out is NULL") : BD_E_INVALID;
    if (window < 0 || window >= ctx->step / ctx->cfg.window_steps)
        return fail(ctx, BD_E_INVALID, "window %lld not completed", (long long)window);
    return deliver(ctx, out, ctx->d_rsf + window * ctx->M, sizeof(double) * ctx->M,
                   is_device_ptr(out));
}

bd_status bd_conformation(bd_ctx* ctx, int64_t window, double* dbar, double* dbead, double* rgz)
{
    if (!ctx) return BD_E_INVALID;
    if (!ctx->conf) return fail(ctx, BD_E_STATE, "created without BD_FLAG_CONFORMATION");
    if (window < 0 || window >= ctx->step / ctx->cfg.window_steps)
        return fail(ctx, BD_E_INVALID, "window %lld not completed", (long long)window);
    bd_status s;
    if (dbar && (s = deliver(ctx, dbar, ctx->d_dbar + window * ctx->n_rep * 3,
                             sizeof(double) * 3 * (size_t)ctx->n_rep, is_device_ptr(dbar))) != BD_OK)
        return s;
    if (dbead && (s = deliver(ctx, dbead, ctx->d_dbead + window * ctx->n_beads * 3,
                              sizeof(double) * 3 * (size_t)ctx->n_beads, is_device_ptr(dbead))) != BD_OK)
        return s;
    if (rgz && (s = deliver(ctx, rgz, ctx->d_rgz + window * ctx->cfg.n_chains,
                            sizeof(double) * (size_t)ctx->cfg.n_chains, is_device_ptr(rgz))) != BD_OK)
        return s;
    return BD_OK;
}

bd_status bd_time_average(bd_ctx* ctx, int64_t window, double* out)
{
    if (!ctx || !out) return ctx ? fail(ctx, BD_E_INVALID, "out is NULL") : BD_E_INVALID;
    if (window < 0 || window >= ctx->step / ctx->cfg.window_steps)
        return fail(ctx, BD_E_INVALID, "window %lld not completed", (long long)window);
    return deliver(ctx, out, ctx->d_tsf + window * ctx->M, sizeof(double) * ctx->M,
                   is_device_ptr(out));
}

bd_status bd_detect_events(bd_ctx* ctx, bd_event* out, int64_t capacity, int64_t* n_out,
                           double* log_surv)
{
    if (!ctx) return BD_E_INVALID;
    if (!n_out) return fail(ctx, BD_E_INVALID, "n_out is NULL");
    if (capacity < 0 || (capacity > 0 && !out))
        return fail(ctx, BD_E_INVALID, "out is NULL with capacity > 0");
    bd_status s = apply_windows(ctx);
    if (s != BD_OK) return s;
    const bool dev = capacity > 0 && is_device_ptr(out);
    const int64_t nblk = event_blocks(ctx->M);
    bd_event* dst = out;
    if (capacity > 0 && !dev) {
        s = ensure_io(ctx, sizeof(bd_event) * (size_t)capacity);
        if (s != BD_OK) return s;
        dst = (bd_event*)ctx->d_io;
    }
    ctx->launches += 3;
    BD_CUDA(ctx, run_events(ctx->d_chains, ctx->d_spring_chain, ctx->M, ctx->d_first_thr,
                            ctx->d_first_bell, ctx->d_evt_scratch, dst, capacity, ctx->stream));
    int64_t total = 0;
    BD_CUDA(ctx, cudaMemcpyAsync(&total, ctx->d_evt_scratch + nblk, sizeof(int64_t),
                                 cudaMemcpyDeviceToHost, ctx->stream));
    BD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (capacity > 0 && !dev)
        BD_CUDA(ctx, cudaMemcpy(out, dst, sizeof(bd_event) * (size_t)std::min(total, capacity),
                                cudaMemcpyDeviceToHost));
    if (log_surv) {
        const bool ldev = is_device_ptr(log_surv);
        double* ld = log_surv;
        const size_t n = sizeof(double) * 3 * (size_t)ctx->cfg.n_chains;
        if (!ldev) {
            s = ensure_io(ctx, n);
            if (s != BD_OK) return s;
            ld = (double*)ctx->d_io;
        }
        ++ctx->launches;
        BD_CUDA(ctx, run_log_survival(ctx->d_chains, ctx->cfg.n_chains, ctx->M, ctx->d_lam, ld,
                                      ctx->stream));
        s = deliver(ctx, log_surv, ld, n, ldev);
        if (s != BD_OK) return s;
    }
    *n_out = total;
    s = check_device_error(ctx);
    if (s != BD_OK) return s;
    if (total > capacity)
        return fail(ctx, BD_E_CAPACITY, "%lld events, capacity %lld", (long long)total,
                    (long long)capacity);
    return BD_OK;
}

bd_status bd_get_kinetics(bd_ctx* ctx, double* hazard, int64_t* first_thr, int64_t* first_bell)
{
    if (!ctx) return BD_E_INVALID;
    bd_status s = apply_windows(ctx);
    if (s != BD_OK) return s;
    const size_t n = 3 * (size_t)ctx->M;
    if (hazard && (s = deliver(ctx, hazard, ctx->d_lam, n * sizeof(double), is_device_ptr(hazard))) != BD_OK) return s;
    if (first_thr && (s = deliver(ctx, first_thr, ctx->d_first_thr, n * sizeof(int64_t), is_device_ptr(first_thr))) != BD_OK) return s;
    if (first_bell && (s = deliver(ctx, first_bell, ctx->d_first_bell, n * sizeof(int64_t), is_device_ptr(first_bell))) != BD_OK) return s;
    return BD_OK;
}

bd_status bd_get_positions(bd_ctx* ctx, int32_t all_slots, double* out, int64_t* step)
{
    if (!ctx) return BD_E_INVALID;
    if (!out) return fail(ctx, BD_E_INVALID, "out is NULL");
    const int64_t nbeads = all_slots ? ctx->n_slot_beads : ctx->n_beads;
    const size_t n = sizeof(double) * 3 * (size_t)nbeads;
    const bool dev = is_device_ptr(out);
    double* dst = out;
    if (!dev) {
        bd_status s = ensure_io(ctx, n);
        if (s != BD_OK) return s;
        dst = (double*)ctx->d_io;
    }
    int64_t npairs = ctx->cfg.n_chains;     // (chain, slot) pairs to convert
    if (all_slots) {
        npairs = 0;
        for (const bd_chain_desc& d : ctx->chains) npairs += d.n_replicas + 1;
    }
    ++ctx->launches;
    BD_CUDA(ctx, run_positions(ctx->f64, ctx->d_chains, all_slots ? ctx->d_pair_all : ctx->d_pair_parent,
                               ctx->cfg.n_chains, npairs, all_slots ? 1 : 0, ctx->d_state, dst,
                               ctx->stream));
    if (step) *step = ctx->step;
    return deliver(ctx, out, dst, n, dev);
}

bd_status bd_set_positions(bd_ctx* ctx, const double* pos, int64_t step)
{
    if (!ctx) return BD_E_INVALID;
    if (!pos) return fail(ctx, BD_E_INVALID, "pos is NULL");
    if (step < 0 || step % ctx->cfg.window_steps != 0)
        return fail(ctx, BD_E_INVALID, "step must be a non-negative multiple of window_steps");
    if (step / ctx->cfg.window_steps > ctx->cfg.max_windows)
        return fail(ctx, BD_E_CAPACITY, "step beyond max_windows");
    bd_status s = reset_kinetics(ctx);
    if (s != BD_OK) return s;
    s = load_positions(ctx, pos);
    if (s != BD_OK) return s;
    ctx->step = step;
    ctx->origin = step;
    ctx->windows_detected = step / ctx->cfg.window_steps;
    return BD_OK;
}

bd_status bd_get_info(bd_ctx* ctx, bd_info* out)
{
    if (!ctx) return BD_E_INVALID;
    if (!out) return fail(ctx, BD_E_INVALID, "out is NULL");
    std::vector<unsigned long long> ov(ctx->cfg.n_chains);
    BD_CUDA(ctx, cudaMemcpyAsync(ov.data(), ctx->d_overext, sizeof(unsigned long long) * ov.size(),
                                 cudaMemcpyDeviceToHost, ctx->stream));
    BD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    int64_t tot = 0;
    for (unsigned long long v : ov) tot += (int64_t)v;
    const bd_status se = check_device_error(ctx);
    if (se != BD_OK) return se;
    out->n_springs = ctx->M;
    out->step = ctx->step;
    out->windows_done = ctx->step / ctx->cfg.window_steps;
    out->overextensions = tot;
    out->device_bytes = (int64_t)ctx->bytes;
    out->kernel_launches = ctx->launches;
    out->n_launch_classes = (int32_t)(ctx->var_classes.size() + ctx->par_classes.size());
    out->precision = ctx->cfg.precision;
    return BD_OK;
}

bd_status bd_enable_timing(bd_ctx* ctx, int32_t enable)
{
    if (!ctx) return BD_E_INVALID;
    ctx->timing = enable != 0;
    return BD_OK;
}

bd_status bd_kernel_times(bd_ctx* ctx, double* ms, int64_t* launches)
{
    if (!ctx) return BD_E_INVALID;
    BD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (ms) { ms[0] = ctx->timed_ms[0]; ms[1] = ctx->timed_ms[1]; }
    if (launches) { launches[0] = ctx->timed_n[0]; launches[1] = ctx->timed_n[1]; }
    ctx->timed_ms[0] = ctx->timed_ms[1] = 0.0;
    ctx->timed_n[0] = ctx->timed_n[1] = 0;
    return BD_OK;
}

bd_status bd_autotune(bd_ctx* ctx, int32_t probe_steps, int32_t force)
{
    if (!ctx) return BD_E_INVALID;
    if (probe_steps < 1) return fail(ctx, BD_E_INVALID, "probe_steps must be >= 1");
    if (ctx->step != 0) return fail(ctx, BD_E_STATE, "bd_autotune must come before the first bd_step");
    const std::pair<int, int> key(ctx->device, ctx->cfg.precision);
    std::vector<double> cost;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end() && !force) cost = it->second;
    }
    if (cost.empty()) {
        bd_status s = autotune_probe(ctx, probe_steps, cost);
        if (s != BD_OK) return s;
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        std::vector<double>& c = g_tune_cache[key];
        if (c.empty()) c.assign(kVariantCodes, 0.0);
        for (int v = 0; v < kVariantCodes; ++v) if (cost[v] > 0) c[v] = cost[v];
        cost = c;
    }
    for (int v = 0; v < kVariantCodes; ++v)
        if (cost[v] > 0) ctx->var_cost[v] = cost[v];
    return replan(ctx);
}

bd_status bd_get_plan(bd_ctx* ctx, int32_t* variant, int32_t* groups, double* cost_ns)
{
    if (!ctx) return BD_E_INVALID;
    std::vector<int32_t> first(ctx->cfg.n_chains, -1);
    for (const ItemDev& it : ctx->h_items)
        if (first[it.chain] < 0) first[it.chain] = it.variant;
    for (int c = 0; c < ctx->cfg.n_chains; ++c) {
        if (variant) variant[c] = first[c];
        if (groups) groups[c] = ctx->h_chains[c].n_groups;
    }
    if (cost_ns) {
        const int* vars = ctx->f64 ? kVariantsF64 : kVariantsF32;
        const int nv = ctx->f64 ? kNumVariantsF64 : kNumVariantsF32;
        for (int t = 0; t < nv; ++t) cost_ns[t] = ctx->var_cost[vars[t]];
    }
    return BD_OK;
}

bd_status bd_adjoint(bd_ctx* ctx, const double* grad_rsf, const double* grad_log_surv,
                     double* grad_params)
{
    if (!ctx) return BD_E_INVALID;
    if (!grad_params) return fail(ctx, BD_E_INVALID, "grad_params is NULL");
    const int64_t K = ctx->cfg.checkpoint_steps, S = ctx->cfg.window_steps, M = ctx->M;
    const int C = ctx->cfg.n_chains;
    if (K <= 0) return fail(ctx, BD_E_STATE, "bd_adjoint needs checkpoint_steps > 0 in the configuration");
    bd_status s = adj_buffers(ctx);
    if (s != BD_OK) return s;
    const int64_t w_lo = ctx->origin / S, w_hi = ctx->step / S;
    BD_CUDA(ctx, cudaMemsetAsync(ctx->d_grad, 0, sizeof(double) * 3 * (size_t)C, ctx->stream));
    if (w_hi > w_lo && (grad_rsf || grad_log_surv)) {
        const int64_t n_w = w_hi - w_lo;
        const size_t gb = sizeof(double) * (size_t)n_w * (size_t)M;
        if (ctx->G_bytes < gb) {
            dfree(ctx, ctx->d_G, ctx->G_bytes);
            ctx->d_G = nullptr;
            ctx->G_bytes = 0;
            if ((s = dalloc(ctx, (void**)&ctx->d_G, gb)) != BD_OK) return s;
            ctx->G_bytes = gb;
        }
        const double* grs = nullptr;
        if (grad_rsf) {
            grs = grad_rsf + w_lo * M;
            if (!is_device_ptr(grad_rsf)) {
                BD_CUDA(ctx, cudaMemcpyAsync(ctx->d_G, grs, gb, cudaMemcpyHostToDevice, ctx->stream));
                grs = ctx->d_G;          // the seed kernel updates it in place
            }
        }
        const double* gls = grad_log_surv;
        if (gls && !is_device_ptr(gls)) {
            BD_CUDA(ctx, cudaMemcpyAsync(ctx->d_gls, gls, sizeof(double) * (size_t)C, cudaMemcpyHostToDevice,
                                         ctx->stream));
            gls = ctx->d_gls;
        }
        ++ctx->launches;
        BD_CUDA(ctx, run_adj_seed(ctx->d_chains, ctx->d_spring_chain, M, ctx->d_rsf, w_lo,
                                  n_w, grs, gls, (int)S, ctx->cfg.dt, ctx->d_G, ctx->stream));
        BD_CUDA(ctx, cudaMemsetAsync(ctx->d_lamP, 0, ctx->tsize * 3 * (size_t)M, ctx->stream));

        AdjParams a;
        std::memset(&a, 0, sizeof(a));
        a.sp = base_params(ctx);
        a.adj = ctx->d_adj;
        a.ckpt = ctx->d_ckpt;
        a.repbuf = ctx->d_repbuf;
        a.state_bonds = ctx->state_bonds;
        a.lamP = ctx->d_lamP;
        a.G = ctx->d_G;
        a.mu_stride = ctx->adj_stride;
        a.w_lo = w_lo;
        a.w_hi = w_hi;
        a.grad = ctx->d_grad;
        const int64_t t_max = (w_hi - 1) * S;           // start of the last window
        const int64_t j_max = (t_max - ctx->origin) / K;
        const int per_cta = kAdjThreads / 32;
        cudaStream_t S0 = ctx->stream, S1 = ctx->adj_stream;
        BD_CUDA(ctx, cudaEventRecord(ctx->ev_init, S0));
        BD_CUDA(ctx, cudaStreamWaitEvent(S1, ctx->ev_init, 0));
        int64_t q = 0;                                  // window batches so far
        for (int64_t j = j_max; j >= 0; --j) {
            // parent states of steps [seg_t0, seg_t0 + n) from checkpoint j,
            // into the segment buffer that segment j + 2 used
            const int sb = (int)(j & 1);
            const int64_t seg_t0 = ctx->origin + j * K;
            const int64_t n = (j == j_max) ? t_max - seg_t0 + 1 : K;
            a.segbuf = ctx->d_seg[sb];
            a.seg_t0 = seg_t0;
            a.ckpt_index = j;
            a.t0 = seg_t0;
            a.n_steps = (int32_t)(n - 1);
            BD_CUDA(ctx, cudaStreamWaitEvent(S0, ctx->ev_seg_free[sb], 0));
            if ((s = adj_parents(ctx, ADJ_PARENT_RECOMPUTE, a, S0)) != BD_OK) return s;
            // windows starting in the segment, in batches from the top down
            // (context stream); after each batch the parent sweeps back over
            // the batch's steps (adjoint stream), overlapping the next batch
            const int64_t wa = seg_t0 / S, wb = std::min(w_hi, (seg_t0 + n - 1) / S + 1);
            for (int64_t b1 = wb; b1 > wa; ++q) {
                const int64_t b0 = std::max(wa, b1 - ctx->rep_batch);
                const int mb = (int)(q & 1);
                a.mu = ctx->d_mu[mb];
                a.mu_w0 = b0;
                a.w_batch0 = b0;
                BD_CUDA(ctx, cudaStreamWaitEvent(S0, ctx->ev_mu_free[mb], 0));
                for (const AdjClass& ac : ctx->adj_classes) {
                    a.items = ctx->d_adj_items + ac.item_begin;
                    a.n_items = ac.item_count;
                    const dim3 grid((unsigned)((ac.item_count + per_cta - 1) / per_cta), (unsigned)(b1 - b0));
                    if ((s = adj_launch(ctx, ADJ_REPLICA_WINDOW, ac.L, grid, &a, S0)) != BD_OK) return s;
                }
                BD_CUDA(ctx, cudaEventRecord(ctx->ev_win[mb], S0));
                BD_CUDA(ctx, cudaStreamWaitEvent(S1, ctx->ev_win[mb], 0));
                const int64_t t_lo = b0 * S, t_hi = std::min(b1 * S, seg_t0 + n);
                AdjParams ab = a;
                ab.t0 = t_lo;
                ab.n_steps = (int32_t)(t_hi - t_lo);
                if ((s = adj_parents(ctx, ADJ_PARENT_BACKWARD, ab, S1)) != BD_OK) return s;
                BD_CUDA(ctx, cudaEventRecord(ctx->ev_mu_free[mb], S1));
                b1 = b0;
            }
            BD_CUDA(ctx, cudaEventRecord(ctx->ev_seg_free[sb], S1));
        }
        BD_CUDA(ctx, cudaEventRecord(ctx->ev_done, S1));
        BD_CUDA(ctx, cudaStreamWaitEvent(S0, ctx->ev_done, 0));
    }
    s = deliver(ctx, grad_params, ctx->d_grad, sizeof(double) * 3 * (size_t)C, is_device_ptr(grad_params));
    if (s != BD_OK) return s;
    BD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return BD_OK;
}

bd_status bd_philox_normals(uint64_t seed, int64_t n, const uint32_t* ctr, int32_t precision,
                            double* out, void* stream)
{
    if (n < 0 || (n > 0 && (!ctr || !out))) return BD_E_INVALID;
    if (precision != BD_PREC_FP32 && precision != BD_PREC_FP64) return BD_E_INVALID;
    if (n == 0) return BD_OK;
    cudaStream_t st = (cudaStream_t)stream;
    StepParams p;
    std::memset(&p, 0, sizeof(p));
    round_keys(seed, p.rk0, p.rk1);
    const bool cdev = is_device_ptr(ctr), odev = is_device_ptr(out);
    uint32_t* dctr = const_cast<uint32_t*>(ctr);
    double* dout = out;
    std::vector<void*> tmp;
    auto cleanup = [&]() { for (void* q : tmp) cudaFree(q); };
    if (!cdev) {
        if (cudaMalloc((void**)&dctr, sizeof(uint32_t) * 4 * n) != cudaSuccess) { cudaGetLastError(); return BD_E_OOM; }
        tmp.push_back(dctr);
        if (cudaMemcpyAsync(dctr, ctr, sizeof(uint32_t) * 4 * n, cudaMemcpyHostToDevice, st) != cudaSuccess) { cleanup(); return BD_E_CUDA; }
    }
    if (!odev) {
        if (cudaMalloc((void**)&dout, sizeof(double) * 3 * n) != cudaSuccess) { cudaGetLastError(); cleanup(); return BD_E_OOM; }
        tmp.push_back(dout);
    }
    cudaError_t e = run_normals(precision == BD_PREC_FP64, n, dctr, p, dout, st);
    if (e == cudaSuccess && !odev)
        e = cudaMemcpyAsync(out, dout, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) { cudaGetLastError(); return BD_E_CUDA; }
    return BD_OK;
}

}  // extern "C"
