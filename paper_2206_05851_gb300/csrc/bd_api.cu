// C ABI of the replica-averaged Brownian-dynamics library (include/bdra.h):
// configuration checks, launch planning, device state, and the stream-ordered
// driving of the parent / replica kernels and the support kernels.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "bd_launch.h"
#include "bd_support.h"

using namespace bdra;

namespace {

struct RepClass {      // one replica-kernel launch: items with the same tile and width
    int L, threads;
    bool paired;       // two replicas per lane (replica2_kernel)
    size_t smem;
    int item_begin, item_count;
};
struct ParClass {      // one parent-kernel launch
    int L, G, threads, grid;
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
    std::vector<RepClass> rep_classes;
    std::vector<ParClass> par_classes;
    uint32_t rk0[10], rk1[10];

    ChainDev* d_chains = nullptr;
    ItemDev* d_items = nullptr;
    int32_t* d_parent_items = nullptr;
    int32_t* d_spring_chain = nullptr;
    int64_t* d_pair_parent = nullptr;   // [n_chains + 1] prefix of 1 per chain
    int64_t* d_pair_all = nullptr;      // [n_chains + 1] prefix of R + 1 per chain
    void* d_state = nullptr;
    void* d_snap = nullptr;
    double* d_part = nullptr;
    double* d_tsf = nullptr;
    double* d_tsf_acc = nullptr;
    double* d_lam = nullptr;
    int64_t* d_first_thr = nullptr;
    int64_t* d_first_bell = nullptr;
    double* d_exp1 = nullptr;
    unsigned long long* d_overext = nullptr;
    int64_t* d_evt_scratch = nullptr;
    void* d_io = nullptr;
    size_t io_bytes = 0;
    size_t bytes = 0;
    std::vector<void*> allocs;
    std::string err;
    int64_t launches = 0;
    bool timing = false;
    struct Timed { int kind; cudaEvent_t a, b; };
    std::vector<Timed> timed;
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
struct TileChoice { int L, G, P, groups, warps; bool paired; double cost; };

// Estimated issue slots per lane-step: one replica per lane ~100 per spring
// plus the halo exchange; two replicas per lane ~140 per spring pair (packed
// float32 arithmetic, per-replica Philox and special functions).
constexpr double kLaneCostOne = 100.0, kLaneCostPair = 140.0, kLaneFixed = 40.0;

TileChoice choose_tile(int N, int R, int wmax, int hint, int layout, bool f64)
{
    TileChoice best{0, 0, 0, 0, 0, false, 1e300};
    for (int pass = 0; pass < 2; ++pass) {
        const bool paired = pass == 1;
        if (paired && (f64 || layout == 1)) continue;
        if (!paired && layout == 2) continue;
        const int* tiles = paired ? kPairTiles : kTiles;
        const int ntiles = paired ? kNumPairTiles : kNumTiles;
        for (int t = 0; t < ntiles; ++t) {
            const int L = tiles[t];
            if (hint && L != hint) continue;
            const int G = (N + L - 1) / L;
            if (G > 32) continue;
            const int P = 32 / G;                  // slots (or slot pairs) per warp
            const int per_warp = paired ? 2 * P : P;
            const int cap = per_warp * wmax;
            const int groups = (R + cap - 1) / cap;
            const int per = (R + groups - 1) / groups;
            const int warps = (per + per_warp - 1) / per_warp;
            const double lane_cost = (paired ? kLaneCostPair : kLaneCostOne) * L + kLaneFixed;
            const double cost = (double)groups * warps * 32 * lane_cost / ((double)R * N);
            if (cost < best.cost - 1e-9) best = {L, G, P, groups, warps, paired, cost};
        }
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
    if (cfg->flags & ~BD_FLAG_IDENTICAL_NOISE) return fail(ctx, BD_E_INVALID, "unknown flags");
    if (cfg->layout_hint < 0 || cfg->layout_hint > 2)
        return fail(ctx, BD_E_INVALID, "layout_hint must be 0, 1 or 2");
    if (cfg->layout_hint == 2 && cfg->precision != BD_PREC_FP32)
        return fail(ctx, BD_E_INVALID, "two replicas per lane needs float32 integration");
    if (cfg->lanes_hint) {
        bool one = false, two = false;
        for (int t = 0; t < kNumTiles; ++t) one |= kTiles[t] == cfg->lanes_hint;
        for (int t = 0; t < kNumPairTiles; ++t) two |= kPairTiles[t] == cfg->lanes_hint;
        if (cfg->layout_hint == 2 ? !two : (cfg->layout_hint == 1 || cfg->precision == BD_PREC_FP64) ? !one : !(one || two))
            return fail(ctx, BD_E_INVALID, "lanes_hint %d is not a compiled tile for this layout",
                        cfg->lanes_hint);
    }
    for (int c = 0; c < cfg->n_chains; ++c) {
        const bd_chain_desc& d = cfg->chains[c];
        if (d.n_beads < 2 || d.n_beads > 512)
            return fail(ctx, BD_E_INVALID, "chain %d: n_beads %d outside [2, 512]", c, d.n_beads);
        if (d.n_replicas < 1 || d.n_replicas > 4096)
            return fail(ctx, BD_E_INVALID, "chain %d: n_replicas %d outside [1, 4096]", c, d.n_replicas);
        if (d.spring != BD_SPRING_HOOKE && d.spring != BD_SPRING_FENE)
            return fail(ctx, BD_E_INVALID, "chain %d: unknown spring law %d", c, d.spring);
        if (d.flow < BD_FLOW_NONE || d.flow > BD_FLOW_PLANAR)
            return fail(ctx, BD_E_INVALID, "chain %d: unknown flow %d", c, d.flow);
        if (!(d.H > 0) || !std::isfinite(d.H)) return fail(ctx, BD_E_INVALID, "chain %d: H must be > 0", c);
        if (d.spring == BD_SPRING_FENE && (!(d.b > 0) || !std::isfinite(d.b)))
            return fail(ctx, BD_E_INVALID, "chain %d: FENE b must be > 0", c);
        if (!std::isfinite(d.rate)) return fail(ctx, BD_E_INVALID, "chain %d: rate not finite", c);
    }
    if (cfg->lanes_hint) {
        for (int c = 0; c < cfg->n_chains; ++c)
            if ((cfg->chains[c].n_beads + cfg->lanes_hint - 1) / cfg->lanes_hint > 32)
                return fail(ctx, BD_E_INVALID, "lanes_hint %d too small for chain %d (N=%d)",
                            cfg->lanes_hint, c, cfg->chains[c].n_beads);
    }
    return BD_OK;
}

bd_status plan(bd_ctx* ctx)
{
    const bd_config& cfg = ctx->cfg;
    const int C = cfg.n_chains;
    const int wmax = (ctx->f64 ? max_threads_f64() : max_threads_f32()) / 32;
    ctx->h_chains.resize(C);
    int64_t bead = 0, slot_bead = 0, bond = 0, spr = 0, part = 0;
    struct Pending { int L, warps; bool paired; ItemDev it; };
    std::vector<Pending> pend;
    std::vector<std::pair<std::pair<int, int>, int>> par;   // ((L, G), chain)
    for (int c = 0; c < C; ++c) {
        const bd_chain_desc& d = ctx->chains[c];
        ChainDev& h = ctx->h_chains[c];
        const TileChoice tc = choose_tile(d.n_beads, d.n_replicas, wmax, cfg.lanes_hint,
                                          cfg.layout_hint, ctx->f64);
        if (!tc.L) return fail(ctx, BD_E_INVALID, "chain %d: no tile fits N=%d", c, d.n_beads);
        h.N = d.n_beads; h.R = d.n_replicas; h.n_groups = tc.groups; h.pad = 0;
        h.bead_off = bead; h.slot_bead_off = slot_bead; h.state_off = bond;
        h.spr_off = spr; h.part_off = part;
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
        int begin = 0;
        for (int g = 0; g < tc.groups; ++g) {
            const int cnt = d.n_replicas / tc.groups + (g < d.n_replicas % tc.groups ? 1 : 0);
            const int per_warp = tc.paired ? 2 * tc.P : tc.P;
            const int warps = (cnt + per_warp - 1) / per_warp;
            pend.push_back({tc.L, warps, tc.paired, ItemDev{c, g, begin, cnt}});
            begin += cnt;
        }
        const int Lp = choose_parent_tile(d.n_beads);
        par.push_back({{Lp, (d.n_beads + Lp - 1) / Lp}, c});
        bead += d.n_beads;
        slot_bead += (int64_t)(d.n_replicas + 1) * d.n_beads;
        bond += (int64_t)(d.n_replicas + 1) * nb;
        spr += nb;
        part += (int64_t)tc.groups * nb;
    }
    ctx->n_beads = bead; ctx->n_slot_beads = slot_bead; ctx->state_bonds = bond;
    ctx->M = spr; ctx->part_stride = part;

    // replica launches: one per (L, warps) class
    std::stable_sort(pend.begin(), pend.end(), [](const Pending& a, const Pending& b) {
        if (a.paired != b.paired) return a.paired < b.paired;
        return a.L != b.L ? a.L < b.L : a.warps < b.warps;
    });
    ctx->h_items.clear();
    ctx->rep_classes.clear();
    for (size_t k = 0; k < pend.size(); ++k) {
        const Pending& q = pend[k];
        const ChainDev& h = ctx->h_chains[q.it.chain];
        const size_t smem = (size_t)q.it.rep_count * (h.N - 1) * ctx->tsize;
        if (ctx->rep_classes.empty() || ctx->rep_classes.back().L != q.L ||
            ctx->rep_classes.back().threads != q.warps * 32 ||
            ctx->rep_classes.back().paired != q.paired) {
            ctx->rep_classes.push_back(RepClass{q.L, q.warps * 32, q.paired, smem, (int)k, 0});
        }
        RepClass& rc = ctx->rep_classes.back();
        rc.item_count++;
        rc.smem = std::max(rc.smem, smem);
        ctx->h_items.push_back(q.it);
    }
    // parent launches: one per (L, G) class, two warps per CTA
    std::stable_sort(par.begin(), par.end());
    ctx->h_parent_items.clear();
    ctx->par_classes.clear();
    for (size_t k = 0; k < par.size(); ++k) {
        const int L = par[k].first.first, G = par[k].first.second;
        if (ctx->par_classes.empty() || ctx->par_classes.back().L != L ||
            ctx->par_classes.back().G != G)
            ctx->par_classes.push_back(ParClass{L, G, 64, 0, (int)k, 0});
        ctx->par_classes.back().item_count++;
        ctx->h_parent_items.push_back(par[k].second);
    }
    for (ParClass& pc : ctx->par_classes) {
        const int per_cta = (pc.threads / 32) * (32 / pc.G);
        pc.grid = (pc.item_count + per_cta - 1) / per_cta;
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
    p.tsf_hist = ctx->d_tsf;
    p.tsf_acc = ctx->d_tsf_acc;
    p.lam = ctx->d_lam;
    p.first_thr = ctx->d_first_thr;
    p.first_bell = ctx->d_first_bell;
    p.exp1 = ctx->d_exp1;
    p.overext = ctx->d_overext;
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
        BD_CUDA(ctx, run_window_criteria(ctx->d_chains, ctx->d_spring_chain, ctx->M, ctx->d_part,
                                         ctx->part_stride, ctx->d_tsf, ctx->windows_detected, done,
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

void drop_timed(bd_ctx* ctx)
{
    for (auto& t : ctx->timed) { cudaEventDestroy(t.a); cudaEventDestroy(t.b); }
    ctx->timed.clear();
}

// Records an event pair around one launch when timing is enabled.
struct TimedLaunch {
    bd_ctx* ctx;
    int kind;
    cudaEvent_t a = nullptr, b = nullptr;
    TimedLaunch(bd_ctx* c, int k) : ctx(c), kind(k)
    {
        if (!ctx->timing) return;
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
            cudaGetLastError();
            a = b = nullptr;
            return;
        }
        cudaEventRecord(a, ctx->stream);
    }
    ~TimedLaunch()
    {
        if (!a) return;
        cudaEventRecord(b, ctx->stream);
        ctx->timed.push_back({kind, a, b});
    }
};

void release(bd_ctx* ctx)
{
    if (!ctx) return;
    if (!ctx->allocs.empty()) cudaStreamSynchronize(ctx->stream);
    drop_timed(ctx);
    for (void* p : ctx->allocs) cudaFree(p);
    ctx->allocs.clear();
    cudaGetLastError();
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
    ctx->tsize = ctx->f64 ? sizeof(double) : sizeof(float);
    round_keys(cfg->seed, ctx->rk0, ctx->rk1);

#define BD_TRY(x) do { s = (x); if (s != BD_OK) goto failed; } while (0)
    {
        cudaError_t e = cudaGetDevice(&ctx->device);
        if (e != cudaSuccess) { cudaGetLastError(); s = fail(ctx, BD_E_CUDA, "no CUDA device: %s", cudaGetErrorString(e)); goto failed; }
    }
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
        BD_TRY(upload(ctx, &ctx->d_spring_chain, spring_chain));
        BD_TRY(upload(ctx, &ctx->d_pair_parent, pair_parent));
        BD_TRY(upload(ctx, &ctx->d_pair_all, pair_all));
        BD_TRY(dalloc(ctx, &ctx->d_state, ctx->tsize * 3 * (size_t)ctx->state_bonds));
        BD_TRY(dalloc(ctx, &ctx->d_snap, ctx->tsize * 3 * (size_t)M * (size_t)ctx->chunk_windows));
        BD_TRY(dalloc(ctx, (void**)&ctx->d_part, sizeof(double) * (size_t)W * (size_t)ctx->part_stride));
        BD_TRY(dalloc(ctx, (void**)&ctx->d_tsf, sizeof(double) * (size_t)W * (size_t)M));
        BD_TRY(dalloc(ctx, (void**)&ctx->d_tsf_acc, sizeof(double) * (size_t)M));
        BD_TRY(dalloc(ctx, (void**)&ctx->d_lam, sizeof(double) * 3 * (size_t)M));
        BD_TRY(dalloc(ctx, (void**)&ctx->d_first_thr, sizeof(int64_t) * 3 * (size_t)M));
        BD_TRY(dalloc(ctx, (void**)&ctx->d_first_bell, sizeof(int64_t) * 3 * (size_t)M));
        BD_TRY(dalloc(ctx, (void**)&ctx->d_exp1, sizeof(double) * 3 * (size_t)M));
        BD_TRY(dalloc(ctx, (void**)&ctx->d_overext, sizeof(unsigned long long) * (size_t)C));
        BD_TRY(dalloc(ctx, (void**)&ctx->d_evt_scratch, sizeof(int64_t) * (size_t)(event_blocks(M) + 1)));
        for (const RepClass& rc : ctx->rep_classes) {
            cudaError_t e = ctx->f64 ? prepare_replica_f64(rc.L, rc.smem, nullptr)
                            : rc.paired ? prepare_replica2_f32(rc.L, rc.smem)
                                        : prepare_replica_f32(rc.L, rc.smem, nullptr);
            if (e != cudaSuccess) {
                cudaGetLastError();
                s = fail(ctx, BD_E_CUDA, "kernel set-up for tile %d (%zu B shared): %s", rc.L,
                         rc.smem, cudaGetErrorString(e));
                goto failed;
            }
        }
        {
            cudaError_t e = run_exp1(ctx->d_chains, ctx->d_spring_chain, M, ctx->rk0[0], ctx->rk1[0],
                                     ctx->d_exp1, ctx->stream);
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
    StepParams p = base_params(ctx);
    int64_t t = ctx->step;
    while (t < t_end) {
        const int64_t w_first = (t + S - 1) / S;
        const int64_t chunk_end = std::min(t_end, (w_first + ctx->chunk_windows) * S);
        p.t0 = t;
        p.n_steps = chunk_end - t;
        p.w_snap0 = w_first;
        for (const ParClass& pc : ctx->par_classes) {
            p.parent_items = ctx->d_parent_items + pc.item_begin;
            p.n_parent_items = pc.item_count;
            p.parent_G = pc.G;
            TimedLaunch tl(ctx, 0);
            BD_CUDA(ctx, ctx->f64 ? launch_parent_f64(pc.L, pc.grid, pc.threads, ctx->stream, p)
                                  : launch_parent_f32(pc.L, pc.grid, pc.threads, ctx->stream, p));
            ++ctx->launches;
        }
        for (const RepClass& rc : ctx->rep_classes) {
            p.items = ctx->d_items + rc.item_begin;
            TimedLaunch tl(ctx, 1);
            BD_CUDA(ctx, ctx->f64 ? launch_replica_f64(rc.L, rc.item_count, rc.threads, rc.smem, ctx->stream, p)
                         : rc.paired ? launch_replica2_f32(rc.L, rc.item_count, rc.threads, rc.smem, ctx->stream, p)
                                     : launch_replica_f32(rc.L, rc.item_count, rc.threads, rc.smem, ctx->stream, p));
            ++ctx->launches;
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
    const bool dev = is_device_ptr(out);
    double* dst = out;
    if (!dev) {
        bd_status s = ensure_io(ctx, sizeof(double) * ctx->M);
        if (s != BD_OK) return s;
        dst = (double*)ctx->d_io;
    }
    ++ctx->launches;
    BD_CUDA(ctx, run_rsf(ctx->d_chains, ctx->d_spring_chain, ctx->M, ctx->d_part, ctx->part_stride,
                         window, dst, ctx->stream));
    return deliver(ctx, out, dst, sizeof(double) * ctx->M, dev);
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
    out->n_springs = ctx->M;
    out->step = ctx->step;
    out->windows_done = ctx->step / ctx->cfg.window_steps;
    out->overextensions = tot;
    out->device_bytes = (int64_t)ctx->bytes;
    out->kernel_launches = ctx->launches;
    out->n_launch_classes = (int32_t)(ctx->rep_classes.size() + ctx->par_classes.size());
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
    double t[2] = {0.0, 0.0};
    int64_t n[2] = {0, 0};
    for (auto& e : ctx->timed) {
        float x = 0.0f;
        if (cudaEventElapsedTime(&x, e.a, e.b) != cudaSuccess) {
            cudaGetLastError();
            drop_timed(ctx);
            return fail(ctx, BD_E_CUDA, "cudaEventElapsedTime failed");
        }
        t[e.kind] += x;
        n[e.kind] += 1;
    }
    drop_timed(ctx);
    if (ms) { ms[0] = t[0]; ms[1] = t[1]; }
    if (launches) { launches[0] = n[0]; launches[1] = n[1]; }
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
