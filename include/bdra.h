/*
 * bdra.h - C ABI of the GB300 library for replica-averaged Brownian dynamics
 * (Kania, Nguyen, Oztekin & Webb, "Replica-Averaging: An algorithm to study
 * mechano-reactive processes for polymers under flow conditions",
 * arXiv 2206.05851).
 *
 * Problem statement (Sec. II): bead-spring chains evolve by the overdamped
 * Langevin update of Eq. 1 under an imposed flow. At every sampling time the
 * parent chain is halted, N_R replicas of it are formed, each with its own
 * random-number stream, evolved for the evolution time S, and the force of
 * every spring (Eq. 4) is sampled once per replica at the end and averaged
 * over the replicas (the replica-averaged spring force, RSF); then the parent
 * continues. The time-averaged (TSF) and instantaneous (ISF) spring forces are
 * the two comparison estimators. Events follow from a force criterion
 * (Sec. I: a threshold rupture force; Sec. III: the Bell rate
 * k = k0 exp(f dx / kT) and the survival exp(-integral of k dt)).
 *
 * Model realised here: bead-spring chains with Hookean or FENE springs
 * F = H Q / (1 - H Q^2/b), the paper's collapsed-chain springs (harmonic with
 * a rest length) and Lennard-Jones cohesion (Sec. II), the coarse-grained vWF
 * chain (supplementary Table S1); free draining (Eq. 2 diagonal diffusion) or
 * with the Rotne-Prager-Yamakawa hydrodynamic interaction (Eqs. 1-3);
 * homogeneous shear (v = gdot z x_hat, Sec. II), uniaxial or planar
 * elongation. Units: kT = 1 and a single-bead diffusivity of 1/4 (the
 * update of Eq. 1 is r += [kappa r + F/4] dt + sqrt(dt/2) xi for free
 * draining); the length unit is the caller's: sqrt(kT/H0) for the FENE
 * chains (time zeta/(4 H0)), the bead radius a for the paper's model (time
 * tau/4, tau = 6 pi eta a^3 / kT).
 *
 * Conventions for every entry point:
 *   - All functions are extern "C", never throw, and return a bd_status.
 *     On failure the context keeps its previous state and bd_last_error()
 *     describes the cause. A NULL context gives BD_E_INVALID.
 *   - Array arguments may be host or device pointers of the context's device;
 *     the library detects which. Device arrays are read or written in stream
 *     order on the context's stream; host arrays are copied synchronously
 *     (the call returns once the data are in place). The caller owns every
 *     array it passes; the context owns all of its device state.
 *   - Layouts: positions are float64 [sum_c N_c][3] (chains in order, beads in
 *     order, x y z). Spring profiles are float64 [M] with
 *     M = sum_c (N_c - 1), chain c's springs starting at sum_{c'<c} (N_c' - 1).
 *   - Noise: Philox4x32-10 (Salmon et al., SC'11) with key = (seed low word,
 *     seed high word); chain = bd_config.chain_id_base + the chain's index in
 *     the context. Eq. 1's normals: counter (bead, j | 0 << 24, step, chain)
 *     for replica slots 2j-1 and 2j (slot 0 is the parent, j = 0; slots
 *     1..R the replicas); the output's 128 bits give six 21-bit uniforms
 *     u = (m + 1/2) 2^-21 (m0..m3 the top 21 bits of words 0..3; m4 the low
 *     11 bits of word 0 above the low 10 bits of word 1; m5 the same of words
 *     2 and 3), Box-Muller on (u0, u1), (u2, u3), (u4, u5) gives six normals,
 *     and the odd slot (and the parent) takes the first three, the even slot
 *     the last three. The Exp(1) thresholds of the Bell first-passage test:
 *     counter (spring, 1 << 24, criterion, chain), E = -ln((x0 + 1/2) 2^-32).
 *     Results therefore do not depend on the launch shape.
 */
#ifndef BDRA_H
#define BDRA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bd_ctx bd_ctx;

typedef enum {
    BD_OK = 0,
    BD_E_INVALID = 1,   /* bad argument or configuration */
    BD_E_CUDA = 2,      /* a CUDA call failed (message in bd_last_error) */
    BD_E_OOM = 3,       /* device allocation failed */
    BD_E_STATE = 4,     /* call not valid in the context's current state */
    BD_E_TIMEOUT = 5,   /* a kernel's bounded wait on the tensor cores gave up (reported by
                           bd_detect_events and bd_get_info, and again by every later call of
                           theirs on the context: the steps run since are invalid) */
    BD_E_CAPACITY = 6   /* output or history capacity exceeded */
} bd_status;

/* BD_SPRING_HARMONIC: the paper's collapsed-chain springs (Sec. II),
 * U = (H/2)(|Q| - r0)^2 with rest length r0 (2a), usually with Lennard-Jones
 * cohesion (lj_u > 0); the sampled spring force is the signed H (|Q| - r0)
 * of Eq. 4. Chains of this law run one replica per lane with the pair forces
 * of all their beads, and have no adjoint. */
/* BD_SPRING_VWF: the coarse-grained vWF chain of the supplementary material
 * (Table S1). Spring i joins beads i and i+1; even springs are A2 domains, a
 * FENE spring in parallel with a harmonic spring, with the signed force
 * vwf_fb x + vwf_fa x / (1 - x^2 / vwf_xmax^2) along the bond (x = |Q| - r0;
 * the denominator floored at s_min and counted as an overextension); odd
 * springs are disulfide bonds, H x. Only the A2 domains take part in the
 * threshold and Bell criteria (their unfolding); the disulfide bonds never
 * have events and their hazard stays 0. Runs on the collapsed-chain (and,
 * with hi_a > 0, hydrodynamic-interaction) kernels; no adjoint. */
enum { BD_SPRING_HOOKE = 0, BD_SPRING_FENE = 1, BD_SPRING_HARMONIC = 2, BD_SPRING_VWF = 3 };
enum { BD_FLOW_NONE = 0, BD_FLOW_SHEAR = 1, BD_FLOW_UNIAXIAL = 2, BD_FLOW_PLANAR = 3 };
/* BD_PREC_FP64: every step in float64. BD_PREC_FP32: Eq. 1 integrated in
 * float32; the cross-replica force reduction and the Bell hazard
 * (log-survival) accumulate in float64. */
enum { BD_PREC_FP64 = 0, BD_PREC_FP32 = 1 };
/* Criterion bits (also the criterion index q = 0, 1, 2 of bd_event). */
enum { BD_CRIT_ISF = 1, BD_CRIT_TSF = 2, BD_CRIT_RSF = 4 };
/* BD_FLAG_IDENTICAL_NOISE: every replica draws the parent's noise (slot 0),
 * so replicas reproduce the parent exactly - a consistency check.
 * BD_FLAG_CONFORMATION: at every window end also compute the conformation
 * diagnostics of Eq. 5 (bd_conformation).
 * BD_FLAG_TEST_TC_STALL: failure test of the tensor-core kernels (float32
 * chains with hydrodynamic interaction of up to 50 beads): they issue no MMA
 * and no completion, so their bounded waits give up (about a second each);
 * the results of such a run are invalid and bd_detect_events / bd_get_info
 * return BD_E_TIMEOUT. No device fault or hang is involved. */
enum { BD_FLAG_IDENTICAL_NOISE = 1, BD_FLAG_CONFORMATION = 2, BD_FLAG_TEST_TC_STALL = 4 };

/* One parent chain with its replica set. */
typedef struct {
    int32_t n_beads;     /* N, 2 <= N <= 512 */
    int32_t n_replicas;  /* N_R, 1 <= N_R <= 4096 */
    int32_t spring;      /* BD_SPRING_* */
    int32_t flow;        /* BD_FLOW_* */
    double H;            /* spring constant in units of H0 (> 0) */
    double b;            /* FENE extensibility H Q0^2 / kT (> 0; unused for Hooke) */
    double rate;         /* shear rate or elongation rate, 1 / (zeta/(4 H0)) */
    double f_c;          /* threshold-rupture force (kT / l_H) */
    double k0;           /* Bell zero-force rate */
    double dx;           /* Bell distance to the transition state (l_H) */
    double r0;           /* BD_SPRING_HARMONIC / BD_SPRING_VWF rest length (>= 0); unused otherwise */
    double lj_u;         /* Lennard-Jones depth between non-adjacent beads, U = lj_u
                            [(s/r)^12 - 2 (s/r)^6] (Sec. II); 0 = none; needs
                            BD_SPRING_HARMONIC or BD_SPRING_VWF */
    double lj_sigma;     /* its minimum distance s (> 0 when lj_u > 0) */
    double hi_a;         /* bead radius a of the Rotne-Prager-Yamakawa hydrodynamic
                            interaction (Eqs. 1-3), in the chain's length unit;
                            0 = free draining. With hi_a > 0: n_beads <= 64 and
                            no adjoint (checkpoint_steps 0); every step of every
                            slot factors the 3N x 3N diffusion tensor (Cholesky)
                            for the correlated noise */
    double vwf_fa;       /* BD_SPRING_VWF: FENE spring constant of the A2 domains (>= 0) */
    double vwf_fb;       /* BD_SPRING_VWF: harmonic spring constant of the A2 domains (>= 0) */
    double vwf_xmax;     /* BD_SPRING_VWF: FENE maximum extension beyond r0 (> 0) */
} bd_chain_desc;

typedef struct {
    int32_t n_chains;             /* >= 1 */
    int32_t window_steps;         /* S / dt: replica evolution time in steps, >= 1 */
    const bd_chain_desc* chains;  /* host array [n_chains], copied by bd_create */
    double dt;                    /* time step (> 0) */
    uint64_t seed;                /* Philox key */
    int32_t precision;            /* BD_PREC_* */
    int32_t flags;                /* BD_FLAG_* */
    int32_t thr_mask;             /* BD_CRIT_* bits with a threshold criterion */
    int32_t bell_mask;            /* BD_CRIT_* bits with a Bell criterion */
    int64_t max_windows;          /* capacity of the per-window profile history */
    double s_min;                 /* FENE floor of 1 - H Q^2 / b (e.g. 1e-3) */
    void* stream;                 /* cudaStream_t for all work; NULL = default stream */
    int32_t lanes_hint;           /* 0: planner's choice; else springs per lane (tile) */
    int32_t layout_hint;          /* 0: planner's choice; 1: one replica per lane;
                                     2: two replicas per lane (float32 only). Both
                                     hints apply to Hooke and FENE chains; harmonic
                                     chains always take the planner's tile */
    int32_t checkpoint_steps;     /* 0: no adjoint; else K, a multiple of window_steps:
                                     bd_step keeps the parent conformation every K
                                     steps so that bd_adjoint can recompute the run */
    int32_t chain_id_base;        /* noise-counter chain word of chain 0 (>= 0): chain c
                                     draws with chain id chain_id_base + c. A workload
                                     split into contiguous chain ranges over several
                                     contexts (one per GPU, Sec. II: the replica sets
                                     are independent simulations) draws, with each
                                     range's first global index here, exactly the noise
                                     of the whole workload in one context. 0 for a
                                     context that holds the whole workload */
} bd_config;

/* A first event of one spring under one criterion. */
typedef struct {
    int32_t chain;      /* chain index */
    int32_t spring;     /* spring index within the chain, 0 .. N-2 */
    int32_t criterion;  /* 0 ISF, 1 TSF, 2 RSF */
    int32_t kind;       /* 0 threshold rupture, 1 Bell first passage */
    int64_t step;       /* global step at which it occurred */
} bd_event;

typedef struct {
    int64_t n_springs;        /* M */
    int64_t step;             /* global step of the parents */
    int64_t windows_done;     /* completed sampling windows */
    int64_t overextensions;   /* FENE-floor applications so far, all slots */
    int64_t device_bytes;     /* device memory held by the context */
    int64_t kernel_launches;  /* CUDA kernels launched by this context so far */
    int32_t n_launch_classes; /* kernel launches per bd_step chunk */
    int32_t precision;
} bd_info;

/* Creates a context on the current CUDA device: validates cfg, plans the
 * launch shapes, allocates the device state and sets every parent to
 * init_pos (float64 [sum N][3], host or device; any frame) at step 0 with its
 * replicas spawned from it. Cites Sec. II (problem set-up). *out receives the
 * context, or NULL on failure. Positions are not checked for finiteness: a
 * NaN or infinite coordinate propagates into that chain's results (other
 * chains are unaffected) and never faults. */
bd_status bd_create(const bd_config* cfg, const double* init_pos, bd_ctx** out);

/* Replica spawn (Sec. II): replicas 1..N_R of every chain <- parent. Also
 * performed automatically by bd_step at the start of every window. */
bd_status bd_spawn_replicas(bd_ctx* ctx);

/* Advances every parent and replica by n_steps Eq. 1 updates (Sec. II),
 * spawning replicas at each window start, sampling RSF (replicas, once at the
 * window end) and TSF/ISF (parent, every step), and updating the ISF
 * criteria. The work runs in chunks of up to 64 windows, each one launch of
 * a CUDA graph (parent kernels, then one persistent replica kernel per step
 * variant), asynchronous on the context's stream. BD_E_CAPACITY if the run
 * would pass max_windows windows. n_steps = 0 is a no-op. */
bd_status bd_step(bd_ctx* ctx, int64_t n_steps);

/* Replica-averaged spring force of one completed window (Sec. II, RSF):
 * out [M] float64 = mean over each chain's replicas of the spring force at the
 * window end, reduced in float64 in a fixed order. */
bd_status bd_replica_average(bd_ctx* ctx, int64_t window, double* out);

/* Conformation diagnostics of one completed window (Eq. 5, Sec. III); needs
 * BD_FLAG_CONFORMATION at bd_create (BD_E_STATE otherwise). With r-hat the
 * bead positions in a chain's centre-of-mass frame and P_c the halted parent
 * the replicas of the window were formed from:
 *   dbar  [sum_c R_c][3]  per replica k (chains in order, replicas 1..R):
 *                         (1/N) sum_i |rhat_i(S, k) - rhat_i(P_c)| per axis;
 *   dbead [sum_c N_c][3]  per bead i: the same difference averaged over the
 *                         chain's replicas (float64 sums in replica order);
 *   rgz   [n_chains]      z contribution to P_c's radius of gyration,
 *                         sqrt((1/N) sum_i zhat_i^2).
 * Computed at every window end by the replica kernels from the bonds (the
 * positions are their prefix sums), in float64. Any pointer may be NULL;
 * host or device arrays. */
bd_status bd_conformation(bd_ctx* ctx, int64_t window, double* dbar, double* dbead, double* rgz);

/* Time-averaged spring force of one completed window (Sec. II, TSF):
 * out [M] float64 = mean of the parent's spring force over the window's steps. */
bd_status bd_time_average(bd_ctx* ctx, int64_t window, double* out);

/* Mechano-reactive events (Sec. I threshold rupture; Sec. III Bell kinetics):
 * applies the TSF and RSF criteria to every window completed since the last
 * call, then writes the first event of every (chain, spring, criterion, kind)
 * seen so far, ordered by chain, spring, criterion, kind, into out[capacity]
 * (host or device), sets *n_out (host) to their number and, if log_surv is not
 * NULL, writes log_surv [n_chains][3] float64 = -sum over springs of the
 * integrated Bell hazard per criterion. Synchronises the stream.
 * BD_E_CAPACITY if there are more than capacity events (*n_out holds the
 * count; out holds the first capacity). */
bd_status bd_detect_events(bd_ctx* ctx, bd_event* out, int64_t capacity, int64_t* n_out,
                           double* log_surv);

/* Kinetic state per criterion q and spring m (after applying pending windows):
 * hazard [3][M] float64 integrated Bell hazard; first_thr / first_bell
 * [3][M] int64 first event step or -1. Any pointer may be NULL. */
bd_status bd_get_kinetics(bd_ctx* ctx, double* hazard, int64_t* first_thr,
                          int64_t* first_bell);

/* Conformations in each chain's centre-of-mass frame (Eq. 5 frame), float64.
 * all_slots = 0: parents, [sum N][3]. all_slots = 1: every slot, chain-major,
 * slot 0 (parent) then replicas 1..N_R, [sum (N_R+1) N][3]. *step (may be
 * NULL) receives the global step. */
bd_status bd_get_positions(bd_ctx* ctx, int32_t all_slots, double* out, int64_t* step);

/* Restart: every parent <- pos (float64 [sum N][3], any frame), replicas
 * spawned from it, global step <- step (a multiple of window_steps), window
 * history and kinetic state cleared. */
bd_status bd_set_positions(bd_ctx* ctx, const double* pos, int64_t step);

/* Counters and sizes (host struct). */
bd_status bd_get_info(bd_ctx* ctx, bd_info* out);

/* Autotuner of the launch shapes (the batching form of the method: chains of
 * uneven bead and replica counts share one persistent launch). For every
 * compiled step variant - springs per lane, one or two replicas per lane -
 * times the persistent replica kernel on this context's chains (a scratch
 * copy of the state, probe_steps steps with no window boundary inside) and
 * records the throughput cost of one warp-step; then re-plans every chain
 * with the measured costs (per chain, the variant that minimises work items
 * x cost per useful bead-step) and rebuilds the step graph. Costs are cached
 * per device and precision for the process; force != 0 measures again. Must
 * be called before the first bd_step (BD_E_STATE otherwise). Synchronises. */
bd_status bd_autotune(bd_ctx* ctx, int32_t probe_steps, int32_t force);

/* The current plan: variant[c] (springs per lane, plus 100 for two replicas
 * per lane, 200 for the collapsed-chain step; 300 for hydrodynamic
 * interaction, one CTA per replica) and groups[c] (work items) per chain,
 * host arrays of n_chains; cost_ns (host, may be NULL) receives the
 * per-warp-step cost of each compiled tile variant, 22 values in the order
 * float32 {4, 7, 10, 13, 16, 104, 107, 202, 204, 205, 207, 216, 5, 6, 8, 9,
 * 11, 12, 14, 15, 105, 106} or 11 values in the order float64 {2, 4, 7, 10,
 * 13, 16, 202, 204, 205, 207, 216}. Any pointer
 * may be NULL. */
bd_status bd_get_plan(bd_ctx* ctx, int32_t* variant, int32_t* groups, double* cost_ns);

/* Kernel timing for measurement tools. Each chunk graph that bd_step launches
 * records CUDA events before its parent kernels, between the parent and
 * replica kernels, and after the replica kernels. enable != 0: after every
 * chunk bd_step waits for those events and accumulates the two intervals
 * (enable = 0 stops; bd_step then never waits). bd_kernel_times
 * synchronises the stream, returns the accumulated device time in
 * milliseconds and the launch counts since the last call (index 0: parent
 * kernels, 1: replica kernels) and resets them. ms and launches are host
 * arrays of 2; either may be NULL. */
bd_status bd_enable_timing(bd_ctx* ctx, int32_t enable);
bd_status bd_kernel_times(bd_ctx* ctx, double* ms, int64_t* launches);

/* Adjoint of the replica-averaged force (Sec. II) and of the Bell survival on
 * it (Sec. III): gradients with respect to each chain's strain rate, FENE b
 * and spring constant H, by reverse-mode differentiation of the discrete
 * Eq. 1 map with the noise held fixed (pathwise derivatives; the gradient of
 * the run that bd_step produced, with the same Philox draws).
 *
 * Objective: L = sum_{w,m} grad_rsf[w][m] RSF_w[m]
 *              + sum_c grad_log_surv[c] log S_c,
 * log S_c = -sum_w sum_{m of c} k0 exp(RSF_w[m] dx) (window_steps dt), the
 * Bell log-survival of chain c under the RSF criterion (whatever bell_mask
 * is). The sums run over the windows completed since the origin - the
 * step of bd_create or of the last bd_set_positions, whose conformation is
 * held fixed - up to the current step; earlier rows of grad_rsf are ignored.
 *   grad_rsf       float64 [windows_done][M] (rows by window index, as
 *                  bd_replica_average numbers them), or NULL;
 *   grad_log_surv  float64 [n_chains], or NULL;
 *   grad_params    float64 [n_chains][3] out: dL/d(rate, b, H); b enters
 *                  through H/b only for FENE springs (0 for Hooke).
 * Host or device arrays. Needs cfg.checkpoint_steps = K > 0 (BD_E_STATE
 * otherwise). Recomputes the parent from its checkpoints K steps at a time
 * and each window's replicas from the recomputed parent (bitwise the forward
 * trajectories), then runs the adjoint recursions backwards: replicas
 * seeded at each window end, their summed sensitivity injected into the
 * parent's adjoint at the window start. The parameter gradients accumulate
 * in the integration precision over blocks of 16 steps and in float64
 * across blocks, lanes and warps. Work buffers (about (K + 1) M and
 * min(K / window_steps, fit) (window_steps + 1) x all-slot bonds states) are
 * allocated on the first call and kept. Synchronises the stream. */
bd_status bd_adjoint(bd_ctx* ctx, const double* grad_rsf, const double* grad_log_surv,
                     double* grad_params);

/* Diagnostic: the three standard normals the integrator draws for each of n
 * (bead, slot | stream << 24, step, chain) quadruples ctr [n][4] under key
 * `seed` (the generator runs on the slot's counter: its replica pair in word
 * 1, see the noise convention above), in the given precision, written as
 * float64 [n][3]. ctr and out may be host or device. Runs on the current
 * device and stream `stream`; synchronises. */
bd_status bd_philox_normals(uint64_t seed, int64_t n, const uint32_t* ctr, int32_t precision,
                            double* out, void* stream);

/* Measurement: the device's throughput for the integrator's dominant work,
 * Philox4x32 rounds (two 32 x 32 -> 64 multiplies and two three-input XORs
 * each), from a kernel of independent round chains at full occupancy on the
 * current device (about 2 ms). *rounds_per_s (host) receives rounds per
 * second for the whole device. The replica step runs 8 rounds per
 * slot-bead-step (the two others are amortised per bead and per step), so
 * 8 x slot-bead-steps/s over this rate is the step's fraction of the
 * multiply-bound ceiling. Runs on `stream`; synchronises. BD_E_INVALID for a
 * NULL pointer, BD_E_OOM / BD_E_CUDA on device failures. */
bd_status bd_probe_philox_rounds(void* stream, double* rounds_per_s);

/* Measured float32 FMA throughput of the current device (no counterpart in
 * the paper: the denominator of the float32 roofline of the RPY Cholesky
 * kernels): independent fused multiply-add chains at full occupancy, no
 * memory traffic (about 5 ms). *flops_per_s (host) receives floating-point
 * operations per second, an FMA counted as two. Runs on `stream`;
 * synchronises. BD_E_INVALID for a NULL pointer, BD_E_OOM / BD_E_CUDA on
 * device failures. */
bd_status bd_probe_fp32_fma(void* stream, double* flops_per_s);

/* The same for float64 FMA (the FP64 path's unit; FLOP/s, an FMA counted as
 * two) and for the special-function unit (approximate reciprocal square
 * roots per second). Same conventions. */
bd_status bd_probe_fp64_fma(void* stream, double* flops_per_s);
bd_status bd_probe_mufu(void* stream, double* ops_per_s);

/* Measured instruction-issue rate of the current device (no counterpart in
 * the paper: the denominator of the issue roofline of the free-draining and
 * collapsed-chain replica kernels, whose work is a mix of integer and
 * float32 instructions): independent chains of two float32 FMAs and one
 * three-input logic operation, full occupancy, no memory traffic (about
 * 5 ms), so that no single pipe but issue binds. *lane_instr_per_s (host)
 * receives thread-instructions per second for the whole device (loop control
 * not counted: low by at most 3%). Same conventions as the probes above. */
bd_status bd_probe_issue(void* stream, double* lane_instr_per_s);

/* Measured integer-ALU throughput (no counterpart in the paper: the unit of
 * the noise fields' bit operations and Philox's XORs): independent chains of
 * three-input logic operations (LOP3), full occupancy, no memory traffic.
 * *ops_per_s (host) receives operations per second for the whole device.
 * Same conventions as the probes above. */
bd_status bd_probe_int_alu(void* stream, double* ops_per_s);

/* Largest n_springs bd_compact_events_noalloc accepts (its fixed scratch
 * holds one count per 256 springs: 32 KiB of device memory). */
#define BD_NOALLOC_MAX_SPRINGS (1 << 20)

/* Event compaction that allocates nothing. (The paper has no counterpart:
 * this is a deployment variant of the event list of bd_detect_events.)
 *
 * Who needs it: callers that may not allocate device memory at the point
 * of the call, such as code running while a CUDA stream is being captured
 * into a graph (where cudaMalloc is not allowed), a host application or
 * engine that owns a fixed device-memory arena and forbids allocation by its
 * plug-ins, or a real-time loop that must not stall on the allocator. It
 * calls no cudaMalloc / cudaFree and no allocating library routine.
 *
 * Input (all device memory of the current device, caller-owned):
 * first_thr / first_bell int64 [3][n_springs] first event steps (-1 = none),
 * as bd_get_kinetics returns them; spring_offsets int64 [n_chains + 1],
 * chain c owning springs spring_offsets[c] .. spring_offsets[c+1]-1.
 * Output (device): out[capacity] receives the events in the order of
 * bd_detect_events (chain, spring, criterion, kind); *n_out (device int64)
 * receives the total number, which may exceed capacity (then only the first
 * capacity records are written). Asynchronous on `stream`.
 *
 * Scratch: a fixed file-scope device array (BD_NOALLOC_MAX_SPRINGS / 256 + 1
 * int64, held by every device that loads the library until exit), shared by
 * every call on a device and overwritten by each; no value from an earlier
 * call is read. Calls that overlap on the GPU (different streams, or
 * different host threads without ordering) race on it and must be
 * serialised by the caller. The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.
 *
 * Errors: BD_E_INVALID for NULL pointers or negative sizes, BD_E_CAPACITY if
 * n_springs > BD_NOALLOC_MAX_SPRINGS, BD_E_CUDA if the look-up or a launch
 * fails. */
bd_status bd_compact_events_noalloc(const int64_t* first_thr, const int64_t* first_bell,
                                    int64_t n_springs, const int64_t* spring_offsets,
                                    int32_t n_chains, bd_event* out, int64_t capacity,
                                    int64_t* n_out, void* stream);

/* Message of the last failure on ctx (never NULL). */
const char* bd_last_error(const bd_ctx* ctx);
/* Name of a status code (never NULL). */
const char* bd_status_string(bd_status s);
/* Releases the context and its device memory; NULL is ignored. */
void bd_destroy(bd_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* BDRA_H */
