#!/usr/bin/env python
"""Benchmark of the replica-averaged Brownian-dynamics hot path on GB300.

Workload: 1024 independent FENE chains, N = 100 beads, b = 100, planar
elongational flow at Wi = 5, 64 replicas per chain re-spawned every 100
steps, dt = 5e-4, FP32 integration with FP64 replica reduction; threshold
(0.9 F_max) and Bell (k0 = 1e-6, dx F_max = 20) criteria on the
replica-averaged force. One bench step = 10^4 integration steps of every
chain and replica (100 windows) plus event detection, so the default
--steps 10 times the whole 10^5-step run. Inputs are synthetic (equilibrium
FENE coils from a seeded generator) and resident in HBM.

Metric: bead-steps/s = chains x replicas x beads x steps / time.

Beside the main line the default run reports the FP64 path on the same
chains, an end-to-end run through the C ABI with host buffers, the batched
uneven (4096 chains) and Bell-kinetics (16384 chains) configurations, the
differentiation workload, the paper's model lines (collapsed chains, RPY,
vWF), each with its roofline, CPU oracle baseline and errors against the
oracle. Under torchrun each rank integrates its contiguous range of one
workload of N x the configuration's chains (weak scaling).

--impl reference times the CPU FP64 oracle (the only reference this method
has) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("bead-steps/s (chains×replicas×beads×steps) FP32 batched vs FP64 plain, "
          "1 GB300")
# Minimal lane-instructions per slot-bead-step of the float32 replica step.
# Two replicas per lane (a noise pair: one Philox4x32-10 output gives both
# replicas' six normals), on an SM with two-wide float32 instructions:
# Philox 17.5 (rounds 3-10 of one call per pair: 8 wide multiplies and 8
# three-input XORs a slot; the split's two XORs and the per-bead table load,
# 1.5 a pair), 7 special-function ops (1.5 log2, 1.5 sqrt, 3 sin/cos, 1
# reciprocal), 18 packed float32 instructions (uniforms 2, Box-Muller 2.5,
# spring law 4, Laplacian 3, update 6.5) and 10 bit/compare ops (the six
# 21-bit uniform fields as float bits, 8; floor clamp and count, 2): 52.5.
# One replica per lane (every float32 operation scalar, one call per slot):
# Philox 35, 8 special-function ops, 36 float32 ops, 12 bit/compare ops (four
# fields, 10 on average over the two halves; floor 2): 91.
OPS_PER_BEAD_STEP_PAIRED = 52.5
OPS_PER_BEAD_STEP_SINGLE = 91.0
# Philox rounds run per slot-bead-step (rounds 1-2 amortise per bead and step)
ROUNDS_PER_BEAD_STEP_PAIRED = 4
ROUNDS_PER_BEAD_STEP_SINGLE = 8
# A generic count of the free-draining bead-step (one unamortised Philox call
# and two Box-Muller pairs per bead-step, about 140 lane-instructions),
# reported for context
GENERIC_OPS_PER_BEAD_STEP = 140.0


def measured_issue_ceiling(sptr):
    """The highest thread-instruction issue rate this GPU has shown in the
    library's probes (independent chains, full occupancy, no memory traffic):
    the mixed float32 / integer stream of bd_probe_issue, and the float32 FMA
    stream of bd_probe_fp32_fma (one instruction per FMA, FLOP/s / 2), which
    issues closer to one warp instruction per scheduler and clock. Returns
    (ceiling, mixed rate, FMA rate)."""
    from paper_2206_05851_gb300 import bdra
    mixed = bdra.bd_probe_issue(sptr)
    fma = bdra.bd_probe_fp32_fma(sptr) / 2.0
    return max(mixed, fma), mixed, fma


def plan_work(ctx, chains):
    """Bead-step-weighted minimal lane-instructions and Philox rounds per
    slot-bead-step of a context's plan (two replicas a lane or one)."""
    variants, _, _ = ctx.plan()
    w = [c.n_replicas * c.n_beads for c in chains]
    paired = [100 <= v < 200 for v in variants]
    tot = float(sum(w))
    ops = sum(wi * (OPS_PER_BEAD_STEP_PAIRED if p else OPS_PER_BEAD_STEP_SINGLE)
              for wi, p in zip(w, paired)) / tot
    rounds = sum(wi * (ROUNDS_PER_BEAD_STEP_PAIRED if p else ROUNDS_PER_BEAD_STEP_SINGLE)
                 for wi, p in zip(w, paired)) / tot
    return ops, rounds, sum(wi for wi, p in zip(w, paired) if p) / tot


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum), each
# from one single-pass ncu capture of the current kernels, reported only at the
# workloads captured: the replica kernel at the default workload and chunk (the
# mean of one bench step's two launches, 64 and 36 windows: mostly the per-group
# FP64 sample rows of the fixed-order reduction, 13 MB a window), the HI replica
# kernel over one 1500-step window of its default workload, and the
# collapsed-chain kernel over its timed 3000 steps (its sample rows still sit in
# L2 when it ends, so they are not in its count).
REPLICA_TRAFFIC_BYTES = (172_927_744 + 853_351_168 + 129_504_768 + 486_531_584) / 2
REPLICA_TRAFFIC_AT = ("fene_1024x_n100_r64_planar_wi5", 10_000, REPLICA_TRAFFIC_BYTES)
# the Bell workload's replica kernel: the mean of one 25 000-step bench step's
# five launches (53, 53, 53, 53 and 38 windows)
BELL_TRAFFIC_BYTES = (894_479_104 + 1_680_933_632 + 889_691_648 + 1_676_391_168 + 885_231_616 +
                      1_674_400_000 + 883_840_000 + 1_673_981_440 + 627_121_920 + 1_027_543_296) / 5
BELL_TRAFFIC_AT = ("fene_16384x_n50_r32_uniaxial_wi10_bell", 25_000, BELL_TRAFFIC_BYTES)
HI_TRAFFIC_BYTES = 5_221_632 + 256
HI_TRAFFIC_AT = ("collapsed_hi_128x_n50_r50_shear30", 1500)
COLLAPSED_TRAFFIC_BYTES = 33_043_456 + 667_904
COLLAPSED_TRAFFIC_AT = ("collapsed_1024x_n50_r50_shear30", 3000)
# Minimal lane-instructions per non-adjacent Lennard-Jones pair of the
# collapsed-chain model, the pair evaluated once, in units of the LJ length s
# (x = s/r): separation 3, r^2 3, reciprocal 1, x^4, x^6, x^8 3, x^8 - x^14 1,
# force on both beads 6; per bead, scaling its position to and its pair force
# from those units, 6.
LJ_PAIR_OPS = 17
LJ_BEAD_OPS = 6
SMS, LANES_PER_CLK_PER_SM, SM_MAX_MHZ = 152, 128, 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--chunk", type=int, default=10_000, help="integration steps per bench step")
    ap.add_argument("--chains", type=int, default=0, help="override the workload's chain count")
    ap.add_argument("--workload", default="planar_1024",
                    choices=["planar_1024", "uneven_4096", "bell_16384"])
    ap.add_argument("--autotune", action="store_true", help="measure step variants first")
    ap.add_argument("--lanes-hint", type=int, default=0,
                    help="force the springs-per-lane tile of the main line (profiling)")
    ap.add_argument("--layout-hint", type=int, default=0,
                    help="force one (1) or two (2) replicas per lane on the main line (profiling)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-conformation", action="store_true")
    ap.add_argument("--no-collapsed", action="store_true")
    ap.add_argument("--no-hi", action="store_true")
    ap.add_argument("--no-vwf", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the uneven-batch and Bell-kinetics lines")
    ap.add_argument("--only-vwf", action="store_true",
                    help="only the vWF line (Table 1 set-up)")
    ap.add_argument("--only-rest", action="store_true",
                    help="only the collapsed chain at rest (mean middle-spring force, RSF spread)")
    ap.add_argument("--only-hi", action="store_true",
                    help="only the hydrodynamic-interaction line (Eqs. 1-3)")
    ap.add_argument("--hi-steps", type=int, default=1500,
                    help="timed steps of the hydrodynamic-interaction line (one window: 1500)")
    ap.add_argument("--only-collapsed", action="store_true",
                    help="only the collapsed-chain line (Sec. II model)")
    ap.add_argument("--only-adjoint", action="store_true",
                    help="time only the differentiation workload (for profiling)")
    ap.add_argument("--adjoint-chains", type=int, default=0, help="override its chain count")
    ap.add_argument("--adjoint-steps", type=int, default=0, help="override its step count")
    return ap.parse_args()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p))
        except Exception:
            return None
    return None


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"bdra_clocks_{os.getpid()}.csv")

    def start(self):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        idx = vis.split(",")[int(os.environ.get("LOCAL_RANK", "0"))] if vis else os.environ.get("LOCAL_RANK", "0")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample
# ---------------------------------------------------------------------------

def cpu_baseline(wl, pos0, n_chains=None, n_steps=1000, sample=None, keep=False):
    """The FP64 oracle timed on the host cores over a bounded sample of the
    workload: the first `n_chains` chains (or the chain indices `sample`),
    `n_steps` steps, OpenMP over chains, with the chains' global ids in the
    noise counter. With keep=True also returns the oracle's results (the
    reference of errors_vs_oracle)."""
    import numpy as np
    from oracle import oracle as O
    from paper_2206_05851_gb300 import inputs as I
    cores = os.cpu_count() or 1
    if sample is None:
        sample = list(range(min(n_chains or cores, wl.n_chains)))
    sub = [wl.chains[c] for c in sample]
    boff = I.bead_offsets(wl.chains)
    sub_pos = np.concatenate([pos0[boff[c]:boff[c + 1]] for c in sample])
    t = time.perf_counter()
    r = O.run(sub, wl.dt, wl.window_steps, n_steps, wl.seed, sub_pos, thr_mask=wl.thr_mask,
              bell_mask=wl.bell_mask, n_threads=min(cores, len(sub)), want_replicas=False,
              chain_ids=list(sample))
    dt = time.perf_counter() - t
    bead_steps = sum(c.n_replicas * c.n_beads for c in sub) * n_steps
    what = (f"first {len(sub)} chains" if list(sample) == list(range(len(sub)))
            else f"{len(sub)} sampled chains {list(sample)[:8]}{'...' if len(sub) > 8 else ''}")
    line = {"value": bead_steps / dt, "unit": "bead-steps/s", "cores": min(cores, len(sub)),
            "kind": "oracle",
            "sample": f"{what} of the workload, {n_steps} steps "
                      f"({bead_steps:.3g} bead-steps, {dt:.1f} s wall, FP64, OpenMP over chains)"}
    return (line, r, sample, sub_pos) if keep else line


def errors_vs_oracle(wl, r, sample, sub_pos, n_steps, sptr):
    """Each result of a float32 GPU run against the FP64 oracle on the sampled
    chains (the CPU baseline's sample and run): a context of those chains,
    with their global chain ids, integrated for the same steps. Positions:
    per-chain max |difference| / max |position| (centre-of-mass frame); RSF
    and TSF: per (chain, window) row, max |difference| / row max |force|;
    Bell log-survival: relative difference per chain and criterion; first
    events: how many steps are equal."""
    import numpy as np
    import torch
    from oracle import oracle as O
    from paper_2206_05851_gb300 import bdra
    from paper_2206_05851_gb300 import inputs as I
    sub = [wl.chains[c] for c in sample]
    contiguous = list(sample) == list(range(sample[0], sample[0] + len(sample)))
    out = {"sample": f"{len(sub)} chains, {n_steps} steps (the CPU baseline's run)"}
    if not contiguous:
        return dict(out, skipped="sample not a contiguous chain range")
    S = wl.window_steps
    nw = n_steps // S
    c = bdra.Context(sub, wl.dt, S, wl.seed, torch.from_numpy(sub_pos).cuda(),
                     precision=bdra.BD_PREC_FP32, max_windows=nw + 1, thr_mask=wl.thr_mask,
                     bell_mask=wl.bell_mask, stream=sptr, chain_id_base=int(sample[0]))
    c.step(n_steps)
    pos = c.positions(False)
    rsf = np.array([c.replica_average(w) for w in range(nw)]).reshape(nw, c.M)
    tsf = np.array([c.time_average(w) for w in range(nw)]).reshape(nw, c.M)
    haz, ft, fb = c.kinetics()
    c.close()
    nb = [ch.n_beads for ch in sub]
    want = O.com_frame(r["pos"], nb)
    boff, soff = I.bead_offsets(sub), I.spring_offsets(sub)

    def rows(g, w):
        worst = 0.0
        for k in range(len(sub)):
            a, b = g[:, soff[k]:soff[k + 1]], w[:, soff[k]:soff[k + 1]]
            worst = max(worst, float((np.abs(a - b).max(axis=1) /
                                      np.maximum(np.abs(b).max(axis=1), 1e-300)).max()))
        return worst

    out["positions_max_rel_err"] = max(
        float(np.abs(pos[boff[k]:boff[k + 1]] - want[boff[k]:boff[k + 1]]).max()
              / np.abs(want[boff[k]:boff[k + 1]]).max()) for k in range(len(sub)))
    if nw:
        out["rsf_max_rel_err"] = rows(rsf, r["rsf"])
        out["tsf_max_rel_err"] = rows(tsf, r["tsf"])
    ls_g = np.array([haz[:, soff[k]:soff[k + 1]].sum(axis=1) for k in range(len(sub))])
    ls_r = np.array([r["lam"][:, soff[k]:soff[k + 1]].sum(axis=1) for k in range(len(sub))])
    on = ls_r > 0
    if on.any():
        out["log_survival_max_rel_err"] = float((np.abs(ls_g - ls_r)[on] / ls_r[on]).max())
    for kind, g, w in (("threshold", ft, r["first_thr"]), ("bell", fb, r["first_bell"])):
        ev = (g >= 0) | (w >= 0)
        out[f"first_{kind}_events"] = {"equal": int(((g == w) & ev).sum()), "total": int(ev.sum())}
    out["precision"] = "GPU float32 integration (FP64 reductions) vs the FP64 oracle, same Philox draws"
    return out


def make_workload(args, world: int = 1):
    """The configuration named by --workload, with world x its chain count
    (one workload that the ranks split)."""
    from paper_2206_05851_gb300 import inputs as I
    make = {"planar_1024": I.planar_1024, "uneven_4096": I.uneven_4096,
            "bell_16384": I.bell_16384}[args.workload]
    if args.chains or world > 1:
        base = args.chains or make().n_chains
        return make(n_chains=base * world)
    return make()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2206_05851_gb300 import inputs as I
    wl = make_workload(args)
    pos0 = I.initial_positions(wl)
    cores = os.cpu_count() or 1
    n_chains = min(cores, wl.n_chains)
    n_steps = 400
    for _ in range(args.warmup):
        cpu_baseline(wl, pos0, n_chains, n_steps)
    vals = [cpu_baseline(wl, pos0, n_chains, n_steps) for _ in range(args.steps)]
    bead_steps = sum(c.n_replicas * c.n_beads for c in wl.chains[:n_chains]) * n_steps
    total_t = sum(bead_steps / v["value"] for v in vals)
    value = bead_steps * len(vals) / total_t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "bead-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total_t / len(vals), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "reference": "CPU FP64 oracle (plain C, OpenMP over chains)",
                       "sample_per_step": f"{n_chains} chains x {n_steps} steps"},
            "cpu_baseline": {"value": value, "unit": "bead-steps/s", "cores": vals[0]["cores"],
                             "kind": "oracle", "sample": vals[0]["sample"]},
            "e2e": {"value": value, "unit": "bead-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def kinetics_summary(first_thr, first_bell, chains, thr_mask, bell_mask, n_steps, dt):
    """First events of the timed run per criterion (ISF, TSF, RSF) and kind
    (threshold, Bell): chains with an event, mean and median first-event step
    (mean first time to unfolding, over the chains that ruptured), and the
    histogram of the rupture location (spring index, or ten bins of relative
    position along the chain when bead counts differ)."""
    import numpy as np
    from paper_2206_05851_gb300 import inputs as I
    offs = I.spring_offsets(chains)
    C = len(chains)
    same_n = len({c.n_beads for c in chains}) == 1
    res = {"timed_steps": n_steps, "dt": dt, "chains": C}
    for q, crit in enumerate(("ISF", "TSF", "RSF")):
        if not ((thr_mask | bell_mask) >> q) & 1:
            continue
        entry = {}
        for kind, arr, mask in (("threshold", first_thr, thr_mask), ("bell", first_bell, bell_mask)):
            if not (mask >> q) & 1:
                continue
            steps = np.full(C, -1, dtype=np.int64)
            loc = np.full(C, -1.0)
            for c in range(C):
                row = arr[q, offs[c]:offs[c + 1]]
                hit = np.nonzero(row >= 0)[0]
                if hit.size:
                    i = hit[np.argmin(row[hit])]
                    steps[c] = row[i]
                    loc[c] = i if same_n else i / max(chains[c].n_beads - 2, 1)
            ok = steps >= 0
            if same_n:
                hist = np.bincount(loc[ok].astype(np.int64), minlength=chains[0].n_beads - 1)
            else:
                hist = np.histogram(loc[ok], bins=10, range=(0.0, 1.0))[0]
            entry[kind] = {"ruptured": int(ok.sum()), "fraction": float(ok.mean()),
                           "mean_first_step": float(steps[ok].mean()) if ok.any() else None,
                           "median_first_step": float(np.median(steps[ok])) if ok.any() else None,
                           "location_hist": hist.tolist()}
        res[crit] = entry
    return res


def replica_line(wl, pos0, base, chunk, steps, warmup, sptr, autotune, issue_peak, philox_peak,
                 dist=None, traffic_at=None, keep_ctx=False, warm_chunk=None, lanes_hint=0,
                 layout_hint=0):
    """Times `steps` bench steps of `chunk` integration steps each, plus event
    detection, of the free-draining workload `wl` (this rank's chains, global
    chain index of the first: `base`), after `warmup` untimed steps of
    `warm_chunk` integration steps, the timed region between barriers and
    synchronisations with L2 flushed between timed steps. Returns the
    whole-job throughput (all ranks' bead-steps over the slowest rank's time)
    and the replica kernel's roofline against the measured issue rate and
    the measured Philox-round ceiling."""
    import numpy as np
    import torch
    from paper_2206_05851_gb300 import bdra, shard
    warm_chunk = warm_chunk or chunk
    S = wl.window_steps
    total_windows = (warmup * warm_chunk + steps * chunk) // S + 1
    stream = torch.cuda.current_stream()
    ctx = bdra.Context(wl.chains, wl.dt, S, wl.seed, torch.from_numpy(pos0).cuda(),
                       precision=bdra.BD_PREC_FP32, max_windows=total_windows,
                       thr_mask=wl.thr_mask, bell_mask=wl.bell_mask, stream=sptr, chain_id_base=base,
                       lanes_hint=lanes_hint, layout_hint=layout_hint)
    if autotune:
        ctx.autotune(probe_steps=32)
    units_chunk = wl.bead_steps(chunk)
    ev_cap = 6 * ctx.M
    ev_buf = torch.zeros(ev_cap * 24, dtype=torch.uint8, device="cuda")
    ls_buf = torch.zeros((len(wl.chains), 3), dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def bench_step(n):
        ctx.step(n)
        return bdra.bd_detect_events(ctx.ptr, ev_buf, ev_cap, ls_buf)

    for _ in range(warmup):
        bench_step(warm_chunk)
    # the timed region integrates the workload itself: from the initial coils at step 0
    ctx.set_positions(torch.from_numpy(pos0).cuda(), 0)
    torch.cuda.synchronize()
    bdra.bd_enable_timing(ctx.ptr, True)
    bdra.bd_kernel_times(ctx.ptr)
    launches0 = ctx.info().kernel_launches
    clocks = ClockSampler()
    clocks.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        flush.zero_()                 # evict L2 between timed steps
        n_events = bench_step(chunk)
    e1.record(stream)
    torch.cuda.synchronize()
    t_ms = e0.elapsed_time(e1)
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    launches = ctx.info().kernel_launches - launches0    # our kernels only
    (par_ms, rep_ms), (par_n, rep_n) = bdra.bd_kernel_times(ctx.ptr)
    bdra.bd_enable_timing(ctx.ptr, False)
    t_max = shard.max_over_ranks(t_ms, dist, "cuda")
    units_all = float(shard.sum_counts(np.array([float(units_chunk * steps)]), dist, "cuda")[0])
    value = shard.whole_job_rate(units_all, t_max / 1e3)

    # roofline of the dominant kernel (replica kernel), measured live
    rep_units = units_chunk * steps
    ops, rounds_per, paired_share = plan_work(ctx, wl.chains)
    achieved = ops * rep_units / (rep_ms / 1e3)
    derived = SMS * LANES_PER_CLK_PER_SM * SM_MAX_MHZ * 1e6
    roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": issue_peak / 1e12,
            "unit": "T lane-instructions/s", "frac": achieved / issue_peak,
            "traffic": traffic_at[2] if traffic_at and (wl.name, chunk) == traffic_at[:2] else None,
            "traffic_unit": "bytes per launch (ncu capture)",
            "kernel": "replica kernel (planner's float32 tile)", "avg_launch_ms": rep_ms / max(rep_n, 1),
            "launches": rep_n, "share_of_step": rep_ms / t_ms,
            "peak_basis": "measured before the timed region: the higher issue rate of the library's "
                          "mixed float32/integer probe (bd_probe_issue) and float32 FMA probe "
                          "(bd_probe_fp32_fma / 2)",
            "peak_derived": derived / 1e12, "frac_of_derived": achieved / derived,
            "ops_per_bead_step": ops, "paired_share": paired_share,
            "ops_basis": f"minimal lane-instructions per slot-bead-step of the plan's layouts "
                         f"({OPS_PER_BEAD_STEP_PAIRED} two replicas a lane, {OPS_PER_BEAD_STEP_SINGLE} one)",
            "frac_at_generic_count": GENERIC_OPS_PER_BEAD_STEP * rep_units / (rep_ms / 1e3) / issue_peak}
    if clk:
        roof["frac_of_derived_at_measured_clock"] = achieved / (SMS * LANES_PER_CLK_PER_SM * clk["sm_mhz"] * 1e6)
    # the same kernel against the measured ceiling of its Philox work
    rounds = rounds_per * rep_units / (rep_ms / 1e3)
    roof_philox = {"bound": "alu (Philox rounds: 32x32->64 multiplies + XOR3)", "achieved": rounds / 1e12,
                   "peak": philox_peak / 1e12, "unit": "T rounds/s", "frac": rounds / philox_peak,
                   "peak_basis": "measured by bd_probe_philox_rounds on this GPU before the timed region",
                   "rounds_per_bead_step": rounds_per}
    out = {"value": value, "unit": "bead-steps/s", "ms_per_step": t_max / steps,
           "config": {"workload": wl.name, "chains_per_gpu": len(wl.chains),
                      "beads": [min(c.n_beads for c in wl.chains), max(c.n_beads for c in wl.chains)],
                      "replicas": sorted({c.n_replicas for c in wl.chains}),
                      "dt": wl.dt, "window_steps": S, "steps_per_bench_step": chunk,
                      "timed_integration_steps": chunk * steps,
                      "criteria": f"threshold mask {wl.thr_mask}, Bell mask {wl.bell_mask} (1 ISF, 2 TSF, 4 RSF)",
                      "precision": "FP32 integrate, FP64 reduce", "autotuned": bool(autotune),
                      "l2": "flushed (256 MB write) between timed steps"},
           "gpu_launches": int(launches), "events_detected_rank": int(n_events),
           "parent_kernel_share": par_ms / t_ms}
    if clk:
        out["clocks"] = clk
    out["roofline"] = roof
    out["roofline_philox"] = roof_philox
    if keep_ctx:
        return out, ctx
    ctx.close()
    return out


def oracle_sample_steps(wl, n_chains, bead_steps=1.0e9):
    """Steps of an oracle sample of the first n_chains chains worth about
    `bead_steps` bead-steps (about 5 s on 16 host cores), whole windows."""
    per_step = sum(c.n_replicas * c.n_beads for c in wl.chains[:n_chains])
    S = wl.window_steps
    return max(S, int(bead_steps / per_step) // S * S)


def batch_line(name, sptr, issue_peak, philox_peak, args):
    """The batched benchmark configurations beside the main one, each its own
    timed run on this GPU, with its kinetics, CPU oracle baseline and errors
    against the oracle:
    - uneven_4096: 4096 chains of 20..500 beads and 8..128 replicas, half in
      shear and half in uniaxial elongation, one persistent launch per step
      variant in one CUDA graph per chunk, shapes picked by the autotuner;
      10^4 steps (the configuration's whole run) in one timed step;
    - bell_16384: 16384 chains of 50 beads, start-up uniaxial elongation at
      Wi = 10 from equilibrium, Bell and threshold criteria on ISF, TSF and
      RSF; 10^5 of the configuration's 2.5 10^5 steps (4 timed steps of
      2.5 10^4), enough for most chains' first rupture; rupture times and
      locations per criterion."""
    from paper_2206_05851_gb300 import inputs as I
    if name == "uneven_4096":
        wl = I.uneven_4096()
        chunk, steps, autotune = 10_000, 1, True
    else:
        wl = I.bell_16384()
        chunk, steps, autotune = 25_000, 4, False
    pos0 = I.initial_positions(wl)
    line, ctx = replica_line(wl, pos0, 0, chunk, steps, 1, sptr, autotune, issue_peak, philox_peak,
                             keep_ctx=True, warm_chunk=1000, traffic_at=BELL_TRAFFIC_AT)
    _, ft, fb = ctx.kinetics()
    ctx.close()
    line["config"]["run"] = (f"{chunk * steps} of the configuration's {wl.n_steps} steps" if
                             chunk * steps < wl.n_steps else "the configuration's whole run")
    line["kinetics"] = kinetics_summary(ft, fb, wl.chains, wl.thr_mask, wl.bell_mask, chunk * steps, wl.dt)
    if not args.no_cpu:
        n_cpu = oracle_sample_steps(wl, 16)
        cpu, r, sample, sub_pos = cpu_baseline(wl, pos0, 16, n_steps=n_cpu, keep=True)
        line["cpu_baseline"] = cpu
        line["errors_vs_oracle"] = errors_vs_oracle(wl, r, sample, sub_pos, n_cpu, sptr)
    return line


def conformation_line(wl, pos0, sptr, n_steps=2000):
    """Cost of the Eq. 5 window-end diagnostics on this workload: the same
    chains integrated n_steps with and without BD_FLAG_CONFORMATION (replica
    kernel time from the chunk graph's events)."""
    import torch
    from paper_2206_05851_gb300 import bdra
    S = wl.window_steps
    times = {}
    for name, flags in (("plain", 0), ("conformation", bdra.BD_FLAG_CONFORMATION)):
        c = bdra.Context(wl.chains, wl.dt, S, wl.seed, torch.from_numpy(pos0).cuda(),
                         precision=bdra.BD_PREC_FP32, max_windows=2 * n_steps // S + 1,
                         thr_mask=wl.thr_mask, bell_mask=wl.bell_mask, flags=flags, stream=sptr)
        c.step(n_steps)                           # warm-up
        c.set_positions(torch.from_numpy(pos0).cuda(), 0)
        bdra.bd_enable_timing(c.ptr, True)
        bdra.bd_kernel_times(c.ptr)
        c.step(n_steps)
        (_, rep_ms), _ = bdra.bd_kernel_times(c.ptr)
        times[name] = rep_ms
        c.close()
    return {"steps": n_steps, "windows": n_steps // S, "replica_ms_plain": times["plain"],
            "replica_ms_conformation": times["conformation"],
            "overhead": times["conformation"] / times["plain"] - 1.0}


def lj_ops_per_bead_step(n_beads):
    """Minimal lane-instructions per bead-step of the collapsed-chain step: the
    noise and bond update of the free-draining step with one replica a lane
    (OPS_PER_BEAD_STEP_SINGLE),
    LJ_BEAD_OPS, and LJ_PAIR_OPS per non-adjacent pair, each pair counted once
    (Newton's third law): (N-1)(N-2)/2 pairs per chain-step."""
    return (OPS_PER_BEAD_STEP_SINGLE + LJ_BEAD_OPS
            + LJ_PAIR_OPS * (n_beads - 1) * (n_beads - 2) / (2.0 * n_beads))


def collapsed_line(sptr, n_chains=0, n_steps=3000, fp64_chains=64, issue_peak=None):
    """The paper's collapsed-chain model (harmonic springs with rest length,
    Lennard-Jones cohesion) on its shear workload: float32 throughput, the
    replica kernel against the issue roofline, the plain FP64 path and the
    FP32 RSF error against it on a subset of the chains, and the CPU oracle
    on a bounded sample."""
    import numpy as np
    import torch
    from paper_2206_05851_gb300 import bdra
    from paper_2206_05851_gb300 import inputs as I

    wl = I.collapsed_1024(**({"n_chains": n_chains} if n_chains else {}))
    pos0 = I.initial_positions(wl)
    S = wl.window_steps
    stream = torch.cuda.current_stream()
    out = {"workload": wl.name, "steps": n_steps, "window_steps": S, "dt": wl.dt}

    def run(chains, p0, prec, steps, timed):
        c = bdra.Context(chains, wl.dt, S, wl.seed, torch.from_numpy(p0).cuda(), precision=prec,
                         max_windows=2 * steps // S + 2, thr_mask=0, bell_mask=0, stream=sptr)
        c.step(S)                                        # warm-up
        c.set_positions(torch.from_numpy(p0).cuda(), 0)
        if timed:
            bdra.bd_enable_timing(c.ptr, True)
            bdra.bd_kernel_times(c.ptr)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        times = bdra.bd_kernel_times(c.ptr) if timed else None
        rsf = [c.replica_average(w) for w in range(steps // S)]
        c.close()
        return t, times, rsf

    t, ((par_ms, rep_ms), (_, rep_n)), _ = run(wl.chains, pos0, bdra.BD_PREC_FP32, n_steps, True)
    units = wl.bead_steps(n_steps)
    out["value"] = units / t
    out["unit"] = "bead-steps/s"
    ops = lj_ops_per_bead_step(wl.chains[0].n_beads)
    achieved = ops * units / (rep_ms / 1e3) / 1e12
    derived = SMS * LANES_PER_CLK_PER_SM * SM_MAX_MHZ * 1e6 / 1e12
    if issue_peak is None:
        issue_peak = measured_issue_ceiling(sptr)[0]     # measured, outside the timed region
    peak = issue_peak / 1e12
    out["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T lane-instructions/s",
                       "frac": achieved / peak, "peak_derived": derived, "frac_of_derived": achieved / derived,
                       "traffic": COLLAPSED_TRAFFIC_BYTES if (wl.name, n_steps) == COLLAPSED_TRAFFIC_AT else None,
                       "traffic_unit": "bytes per launch (ncu capture)",
                       "kernel": "collapsed-chain replica kernel (float32)",
                       "avg_launch_ms": rep_ms / max(rep_n, 1), "launches": rep_n,
                       "share_of_step": rep_ms / (t * 1e3), "ops_per_bead_step": ops,
                       "peak_basis": "measured: the higher issue rate of bd_probe_issue and bd_probe_fp32_fma / 2"}
    out["parent_kernel_share"] = par_ms / (t * 1e3)
    # FP64 and the FP32 force error on a subset
    sub = wl.chains[:fp64_chains]
    psub = pos0[:sum(c.n_beads for c in sub)]
    t64, _, r64 = run(sub, psub, bdra.BD_PREC_FP64, S, False)
    _, _, r32 = run(sub, psub, bdra.BD_PREC_FP32, S, False)
    out["fp64_plain"] = {"value": sum(c.n_replicas * c.n_beads for c in sub) * S / t64,
                         "unit": "bead-steps/s", "sample": f"first {len(sub)} chains, {S} steps",
                         "rsf_max_rel_err_fp32_vs_fp64":
                             float(max(np.abs(a - b).max() / np.abs(b).max() for a, b in zip(r32, r64)))}
    # CPU oracle on a bounded sample
    from oracle import oracle as O
    cores = os.cpu_count() or 1
    sub = wl.chains[:cores]
    psub = pos0[:sum(c.n_beads for c in sub)]
    n_cpu = 20000          # about 10-15 s of oracle work on 16 cores
    tc = time.perf_counter()
    O.run(sub, wl.dt, S, n_cpu, wl.seed, psub, thr_mask=0, bell_mask=0, n_threads=cores,
          want_replicas=False, chain_ids=list(range(len(sub))))
    tc = time.perf_counter() - tc
    bs = sum(c.n_replicas * c.n_beads for c in sub) * n_cpu
    out["cpu_baseline"] = {"value": bs / tc, "unit": "bead-steps/s", "cores": cores, "kind": "oracle",
                           "sample": f"first {len(sub)} chains, {n_cpu} steps ({tc:.1f} s wall, FP64)"}
    return out


def hi_flops_per_slot_step(n_beads):
    """Floating-point operations of one hydrodynamic-interaction step of one
    slot, counting an FMA as two: Cholesky of the 3N x 3N tensor (n^3/3), the
    drift W F with the full symmetric tensor (2 n^2) and the noise L xi (n^2);
    the tensor's assembly, forces and update are O(n^2) or less and not
    counted."""
    n = 3 * n_beads
    return n ** 3 / 3.0 + 2.0 * n * n + n * n


def hi_tc_flops_per_slot_step(n_beads):
    """Floating-point operations the tensor cores execute per slot-step in the
    float32 factorisation of chains of up to 50 beads (an FMA as two): the
    trailing block T (the last 3N - t0 <= 126 rows, t0 = 3 max(0, N - 42)) is
    updated as M = 128 rows x N columns x K MMAs, three tf32 products per
    float32 product; after the head (K = t0 rounded up to 8) and after every
    32-column panel but the last (K = 32), over the next panel's 32 columns
    and the rest of the 16-column-padded width."""
    hb = max(0, n_beads - 42)
    t0 = 3 * hb
    m = 3 * n_beads - t0
    width = (m + 15) // 16 * 16
    panels = (m + 31) // 32
    flops = 0.0
    if t0 > 0:
        flops += 3 * 2 * 128 * max(width, 32) * (8 * ((t0 + 7) // 8))
    for pn in range(panels - 1):
        c1 = 32 * (pn + 1)
        flops += 3 * 2 * 128 * (32 + max(0, width - c1 - 32)) * 32
    return flops


def tf32_peak_tflops():
    """Dense tf32 tensor peak: the measured bf16 GEMM rate (MEASURED_PEAKS.json,
    burst) times the nominal tf32 / bf16 ratio 1.1 / 2.25."""
    mp = measured_peaks()
    return (mp.get("bf16_tflops") or 1900.0) * (1.1 / 2.25)


def hi_tensor_roofline(n_beads, slot_steps, rep_ms):
    """The tensor-core part of the float32 factorisation: the tf32 flops the
    MMAs execute (hi_tc_flops_per_slot_step, six to seven times the useful
    trailing-update flops: three products, the full square, padding) per second
    of the replica kernel against the dense tf32 peak."""
    if n_beads > 50:
        return None
    ach = hi_tc_flops_per_slot_step(n_beads) * slot_steps / (rep_ms / 1e3) / 1e12
    peak = tf32_peak_tflops()
    return {"achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "flops_per_slot_step": hi_tc_flops_per_slot_step(n_beads),
            "peak_basis": "measured bf16 GEMM (MEASURED_PEAKS.json) x nominal tf32/bf16 1.1/2.25"}


def hi_line(sptr, n_chains=0, n_steps=1500, fp64_chains=8, fp64_steps=100):
    """The paper's full model with RPY hydrodynamic interaction: float32
    throughput of one evolution window, the replica kernel against the float32
    FMA peak, the FP64 path and the FP32 RSF error against it on a few chains,
    and the CPU oracle on a bounded sample."""
    import numpy as np
    import torch
    from paper_2206_05851_gb300 import bdra
    from paper_2206_05851_gb300 import inputs as I

    wl = I.collapsed_hi_128(**({"n_chains": n_chains} if n_chains else {}))
    pos0 = I.initial_positions(wl)
    S = wl.window_steps
    stream = torch.cuda.current_stream()
    out = {"workload": wl.name, "steps": n_steps, "window_steps": S, "dt": wl.dt}

    def run(chains, p0, prec, steps, timed, window):
        c = bdra.Context(chains, wl.dt, window, wl.seed, torch.from_numpy(p0).cuda(), precision=prec,
                         max_windows=2 * steps // window + 2, thr_mask=0, bell_mask=0, stream=sptr)
        c.step(min(window, 10))                          # warm-up
        c.set_positions(torch.from_numpy(p0).cuda(), 0)
        if timed:
            bdra.bd_enable_timing(c.ptr, True)
            bdra.bd_kernel_times(c.ptr)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        times = bdra.bd_kernel_times(c.ptr) if timed else None
        rsf = [c.replica_average(w) for w in range(steps // window)]
        c.close()
        return t, times, rsf

    t, ((par_ms, rep_ms), (_, rep_n)), _ = run(wl.chains, pos0, bdra.BD_PREC_FP32, n_steps, True, S)
    units = wl.bead_steps(n_steps)
    out["value"] = units / t
    out["unit"] = "bead-steps/s"
    N = wl.chains[0].n_beads
    slot_steps = sum(c.n_replicas for c in wl.chains) * n_steps
    achieved = hi_flops_per_slot_step(N) * slot_steps / (rep_ms / 1e3) / 1e12
    derived = 2.0 * SMS * LANES_PER_CLK_PER_SM * SM_MAX_MHZ * 1e6 / 1e12
    peak = bdra.bd_probe_fp32_fma(sptr) / 1e12           # measured, outside the timed region
    out["roofline"] = {"bound": "alu (float32 FMA)", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                       "frac": achieved / peak,
                       "traffic": HI_TRAFFIC_BYTES if (wl.name, n_steps) == HI_TRAFFIC_AT else None,
                       "traffic_unit": "bytes per launch (ncu capture)",
                       "kernel": "hydrodynamic-interaction replica kernel (float32, one CTA per replica)",
                       "avg_launch_ms": rep_ms / max(rep_n, 1), "launches": rep_n,
                       "share_of_step": rep_ms / (t * 1e3), "flops_per_slot_step": hi_flops_per_slot_step(N),
                       "peak_basis": "measured by bd_probe_fp32_fma on this GPU after the timed region",
                       "peak_derived": derived, "frac_of_derived": achieved / derived,
                       "tensor": hi_tensor_roofline(N, slot_steps, rep_ms)}
    out["parent_kernel_share"] = par_ms / (t * 1e3)
    # FP64 and the FP32 force error on a few chains (a short window so that
    # RSF samples exist)
    sub = wl.chains[:fp64_chains]
    psub = pos0[:sum(c.n_beads for c in sub)]
    w_short = fp64_steps // 2
    t64, _, r64 = run(sub, psub, bdra.BD_PREC_FP64, fp64_steps, False, w_short)
    _, _, r32 = run(sub, psub, bdra.BD_PREC_FP32, fp64_steps, False, w_short)
    out["fp64_plain"] = {"value": sum(c.n_replicas * c.n_beads for c in sub) * fp64_steps / t64,
                         "unit": "bead-steps/s",
                         "sample": f"first {len(sub)} chains, {fp64_steps} steps, window {w_short}",
                         "rsf_max_rel_err_fp32_vs_fp64":
                             float(max(np.abs(a - b).max() / np.abs(b).max() for a, b in zip(r32, r64)))}
    from oracle import oracle as O
    cores = os.cpu_count() or 1
    sub = wl.chains[:cores]
    psub = pos0[:sum(c.n_beads for c in sub)]
    n_cpu = 600          # about 10 s of oracle work on 16 cores
    s_cmp = 100          # windows of the comparison run (RSF rows to compare)
    tc = time.perf_counter()
    r = O.run(sub, wl.dt, s_cmp, n_cpu, wl.seed, psub, thr_mask=0, bell_mask=0, n_threads=cores,
              want_replicas=False, chain_ids=list(range(len(sub))))
    tc = time.perf_counter() - tc
    bs = sum(c.n_replicas * c.n_beads for c in sub) * n_cpu
    out["cpu_baseline"] = {"value": bs / tc, "unit": "bead-steps/s", "cores": cores, "kind": "oracle",
                           "sample": f"first {len(sub)} chains, {n_cpu} steps in windows of {s_cmp} "
                                     f"({tc:.1f} s wall, FP64)"}
    # the float32 tensor-core path on the same chains, windows and steps
    import dataclasses
    cmp_wl = dataclasses.replace(wl, chains=list(sub), window_steps=s_cmp, thr_mask=0, bell_mask=0)
    out["errors_vs_oracle"] = errors_vs_oracle(cmp_wl, r, list(range(len(sub))), psub, n_cpu, sptr)
    return out


def vwf_line(sptr, n_chains=0, windows=4):
    """The coarse-grained vWF chain at rest with hydrodynamic interaction
    (Table 1's set-up: 50 beads, N_R = 40, S = 0.015 tau): float32 throughput,
    and the mean first time to unfold any A2 domain (MFTU) that the ISF, TSF
    and RSF hazards of the run predict, 1 / (summed A2 unfolding rate per
    chain), in seconds; with the run's mean A2 force."""
    import numpy as np
    import torch
    from paper_2206_05851_gb300 import bdra
    from paper_2206_05851_gb300 import inputs as I

    wl = I.vwf_64(**({"n_chains": n_chains} if n_chains else {}))
    pos0 = I.initial_positions(wl)
    S = wl.window_steps
    n = windows * S
    stream = torch.cuda.current_stream()
    c = bdra.Context(wl.chains, wl.dt, S, wl.seed, torch.from_numpy(pos0).cuda(),
                     precision=bdra.BD_PREC_FP32, max_windows=windows + 2, thr_mask=0,
                     bell_mask=I.CRIT_ALL, stream=sptr)
    c.step(10)                                           # warm-up
    c.set_positions(torch.from_numpy(pos0).cuda(), 0)
    bdra.bd_enable_timing(c.ptr, True)
    bdra.bd_kernel_times(c.ptr)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    c.step(n)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    (par_ms, rep_ms), (_, rep_n) = bdra.bd_kernel_times(c.ptr)
    haz, _, _ = c.kinetics()
    rsf = np.array([c.replica_average(w) for w in range(windows)])
    tsf = np.array([c.time_average(w) for w in range(windows)])
    c.close()
    offs = I.spring_offsets(wl.chains)
    a2 = np.concatenate([np.arange(offs[k], offs[k + 1], 2) for k in range(len(wl.chains))])
    T = n * wl.dt
    C = len(wl.chains)
    mftu = {crit: I.vwf_mftu_seconds(haz[q, a2].sum() / (C * T))
            for q, crit in enumerate(("ISF", "TSF", "RSF"))}
    N = wl.chains[0].n_beads
    slot_steps = sum(ch.n_replicas for ch in wl.chains) * n
    achieved = hi_flops_per_slot_step(N) * slot_steps / (rep_ms / 1e3) / 1e12
    peak = bdra.bd_probe_fp32_fma(sptr) / 1e12           # measured, outside the timed region
    from oracle import oracle as O
    cores = os.cpu_count() or 1
    sub = wl.chains[:cores]
    psub = pos0[:sum(ch.n_beads for ch in sub)]
    n_cpu = 300
    s_cmp = 100          # windows of the comparison run (RSF rows to compare)
    tc = time.perf_counter()
    r = O.run(sub, wl.dt, s_cmp, n_cpu, wl.seed, psub, thr_mask=0, bell_mask=I.CRIT_ALL, n_threads=cores,
              want_replicas=False, chain_ids=list(range(len(sub))))
    tc = time.perf_counter() - tc
    bs = sum(ch.n_replicas * ch.n_beads for ch in sub) * n_cpu
    # the float32 tensor-core path on the same chains, windows and steps
    import dataclasses
    cmp_wl = dataclasses.replace(wl, chains=list(sub), window_steps=s_cmp, thr_mask=0, bell_mask=I.CRIT_ALL)
    ev = errors_vs_oracle(cmp_wl, r, list(range(len(sub))), psub, n_cpu, sptr)
    return {"workload": wl.name, "steps": n, "windows": windows, "window_steps": S,
            "value": wl.bead_steps(n) / t, "unit": "bead-steps/s",
            "roofline": {"bound": "alu (float32 FMA)", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "hydrodynamic-interaction replica kernel (float32)",
                         "share_of_step": rep_ms / (t * 1e3), "launches": rep_n,
                         "peak_basis": "measured by bd_probe_fp32_fma",
                         "tensor": hi_tensor_roofline(N, slot_steps, rep_ms)},
            "parent_kernel_share": par_ms / (t * 1e3),
            "cpu_baseline": {"value": bs / tc, "unit": "bead-steps/s", "cores": cores, "kind": "oracle",
                             "sample": f"first {len(sub)} chains, {n_cpu} steps in windows of {s_cmp} "
                                       f"({tc:.1f} s wall, FP64)"},
            "errors_vs_oracle": ev,
            "precision": "FP32 integrate, FP64 reduce and hazards",
            "mftu_s": mftu,
            "mean_a2_force_pN": {"RSF": float(rsf[:, a2].mean() * I.VWF_FORCE_UNIT_PN),
                                 "TSF": float(tsf[:, a2].mean() * I.VWF_FORCE_UNIT_PN)},
            "paper_table1_context_s": {"ISF": 1.82e-5, "TSF S=0.015": 0.42, "RSF N_R=40 S=0.015": 13.22},
            "start": "compact globules (not equilibrated), run of windows x S from step 0"}


def rest_line(sptr, n_chains=128, windows=6, skip=2):
    """The paper's collapsed chain with hydrodynamic interaction at rest
    (Fig. 1-2 set-up: N = 50, S = 0.02 tau = 2000 steps): the mean force of
    the middle (25th) spring and the spread of its RSF for N_R = 10 and 50,
    over chains and windows after the first `skip` windows (context for the
    paper's 0.55 and 6.7 / 3.3; float32)."""
    import numpy as np
    import torch
    from paper_2206_05851_gb300 import bdra
    from paper_2206_05851_gb300 import inputs as I

    S = 2000
    out = {"chains": n_chains, "window_steps": S, "windows": windows, "skipped_windows": skip}
    for R in (10, 20, 40, 50):
        chains = []
        for _ in range(n_chains):
            ch = I.collapsed_chain(R, rate=0.0)
            ch.hi_a = 1.0
            chains.append(ch)
        wl = I.custom(chains, I.COLLAPSED_DT, S, windows * S)
        pos0 = I.initial_positions(wl, seed=12)
        c = bdra.Context(chains, wl.dt, S, 12, torch.from_numpy(pos0).cuda(), precision=bdra.BD_PREC_FP32,
                         max_windows=windows + 1, stream=sptr)
        t0 = time.perf_counter()
        c.step(windows * S)
        rsf = np.array([c.replica_average(w) for w in range(windows)])
        tsf = np.array([c.time_average(w) for w in range(windows)])
        t = time.perf_counter() - t0
        c.close()
        mid = I.spring_offsets(chains)[:-1] + 24
        r = rsf[skip:, mid]
        out[f"N_R={R}"] = {"rsf_mean": float(r.mean()), "rsf_std": float(r.std()),
                           "tsf_mean": float(tsf[skip:, mid].mean()), "seconds": t}
    # Fig. 2: the TSF of the same spring needs a longer sampling time for the
    # same spread (the paper: S = 0.07 tau for N_R = 10, 0.36 tau for N_R = 50)
    tsf_spread = {}
    for s_tau in (0.02, 0.07, 0.36):
        St = int(round(s_tau * 1e5))                     # steps of 1e-5 tau
        chains = []
        for _ in range(n_chains):
            ch = I.collapsed_chain(1, rate=0.0)
            ch.hi_a = 1.0
            chains.append(ch)
        nw = 3
        pos0 = I.initial_positions(I.custom(chains, I.COLLAPSED_DT, St, nw * St), seed=12)
        c = bdra.Context(chains, I.COLLAPSED_DT, St, 12, torch.from_numpy(pos0).cuda(),
                         precision=bdra.BD_PREC_FP32, max_windows=nw, stream=sptr)
        c.step(nw * St)
        tsf = np.array([c.time_average(w) for w in range(1, nw)])
        c.close()
        mid = I.spring_offsets(chains)[:-1] + 24
        tsf_spread[f"S={s_tau}"] = float(tsf[:, mid].std())
    out["tsf_spread_vs_S"] = tsf_spread
    # Fig. 6 set-up: shear at 30 / tau, N_R = 50, S = 0.015 tau; replica-vs-parent D-bar (Eq. 5)
    chains = []
    for _ in range(64):
        ch = I.collapsed_chain(50)
        ch.hi_a = 1.0
        chains.append(ch)
    S6, w6 = 1500, 3
    wl = I.custom(chains, I.COLLAPSED_DT, S6, w6 * S6)
    pos0 = I.initial_positions(wl, seed=13)
    c = bdra.Context(chains, wl.dt, S6, 13, torch.from_numpy(pos0).cuda(), precision=bdra.BD_PREC_FP32,
                     max_windows=w6, flags=bdra.BD_FLAG_CONFORMATION, stream=sptr)
    c.step(w6 * S6)
    conf = [c.conformation(w) for w in range(1, w6)]
    c.close()
    dbar = np.concatenate([x[0] for x in conf])          # [replicas x windows][3]
    rgz = np.concatenate([x[2] for x in conf])
    out["shear30_eq5"] = {"windows_used": w6 - 1, "dbar_max": dbar.max(axis=0).tolist(),
                          "dbar_mean": dbar.mean(axis=0).tolist(), "rgz_mean": float(rgz.mean()),
                          "rgz_max": float(rgz.max())}
    out["rsf_spread_reduction"] = {"N_R 10->20": out["N_R=20"]["rsf_std"] / out["N_R=10"]["rsf_std"] - 1,
                                   "N_R 20->40": out["N_R=40"]["rsf_std"] / out["N_R=20"]["rsf_std"] - 1}
    out["paper_context"] = {"mean_force_spring25": 0.55, "rsf_std_S0.02": {"N_R=10": 6.7, "N_R=50": 3.3},
                            "rsf_spread_reduction": {"N_R 10->20": -0.27, "N_R 20->40": -0.24},
                            "tsf_S_matching_rsf": {"N_R=10": 0.07, "N_R=50": 0.36},
                            "max_dbar_x_S0.015": 0.65}
    return out


def adjoint_line(sptr, n_chains=0, n_steps=0, grad_check=False):
    """Forward run plus reverse-mode adjoint of the differentiation workload
    (256 FENE chains, N=200, 32 replicas, 2e4 steps, parent checkpoints every
    1000 steps, float32 integration): gradients of the mid-chain RSF averaged
    over the windows plus the Bell log-survival w.r.t. (rate, b, H)."""
    import numpy as np
    import torch
    from paper_2206_05851_gb300 import bdra
    from paper_2206_05851_gb300 import inputs as I

    kw = {}
    if n_chains:
        kw["n_chains"] = n_chains
    if n_steps:
        kw["n_steps"] = n_steps
    wl = I.adjoint_256(**kw)
    pos0 = torch.from_numpy(I.initial_positions(wl)).cuda()
    S, n = wl.window_steps, wl.n_steps
    W = n // S
    offs = I.spring_offsets(wl.chains)
    G = np.zeros((W, int(offs[-1])))
    for c, ch in enumerate(wl.chains):
        G[:, offs[c] + (ch.n_beads - 1) // 2] = 1.0 / W
    G = torch.from_numpy(G).cuda()
    gls = torch.ones(len(wl.chains), dtype=torch.float64, device="cuda")
    grad = torch.empty((len(wl.chains), 3), dtype=torch.float64, device="cuda")
    ctx = bdra.Context(wl.chains, wl.dt, S, wl.seed, pos0, precision=bdra.BD_PREC_FP32,
                       max_windows=W, bell_mask=I.CRIT_RSF, stream=sptr,
                       checkpoint_steps=I.ADJOINT_CHECKPOINT_STEPS)
    warm = min(I.ADJOINT_CHECKPOINT_STEPS, n)
    ctx.step(warm)                                  # warm-up; allocates the work buffers
    bdra.bd_adjoint(ctx.ptr, len(wl.chains), ctx.M, warm // S, G, gls, grad)
    ctx.set_positions(pos0, 0)
    stream = torch.cuda.current_stream()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize()
    e[0].record(stream)
    ctx.step(n)
    e[1].record(stream)
    bdra.bd_adjoint(ctx.ptr, len(wl.chains), ctx.M, W, G, gls, grad)
    e[2].record(stream)
    torch.cuda.synchronize()
    fwd, adj = e[0].elapsed_time(e[1]) / 1e3, e[1].elapsed_time(e[2]) / 1e3
    info = ctx.info()
    ctx.close()
    bead_steps = wl.bead_steps()
    out = {"workload": wl.name, "precision": "FP32 integrate, FP64 reduce",
           "checkpoint_steps": I.ADJOINT_CHECKPOINT_STEPS, "steps": n,
           "forward_s": fwd, "adjoint_s": adj, "adjoint_over_forward": adj / fwd,
           "value": bead_steps / (fwd + adj), "unit": "bead-steps/s (forward + adjoint)",
           "device_bytes": int(info.device_bytes),
           "grad_finite": bool(torch.isfinite(grad).all().item())}
    # HBM roofline of the adjoint's stored replica states: every window's S + 1
    # states of every slot's bonds (float32 x 3) written once by the
    # replica-window kernel's forward sweep and read back once by its backward
    # sweep; over the whole adjoint call (the replica-window kernel is about 84%
    # of the adjoint's launch time in profiles/adjoint_fene256_n200_r32.md, so
    # the kernel's own rate is higher)
    slot_bonds = sum((ch.n_replicas + 1) * (ch.n_beads - 1) for ch in wl.chains)
    stream_bytes = 2.0 * W * (S + 1) * slot_bonds * 3 * 4
    mp = measured_peaks() or {}
    hbm = mp.get("hbm_gbs") or 6800.0
    out["roofline"] = {"bound": "hbm", "achieved": stream_bytes / adj / 1e9, "peak": hbm, "unit": "GB/s",
                       "frac": stream_bytes / adj / 1e9 / hbm, "traffic": None,
                       "bytes_per_adjoint": stream_bytes,
                       "kernel": "adjoint call (replica-window kernel: forward recompute storing the states, "
                                 "backward sweep over them)",
                       "peak_basis": "measured copy bandwidth (MEASURED_PEAKS.json)" if mp.get("hbm_gbs")
                                     else "fallback 6.8 TB/s"}
    if grad_check:
        ev = adjoint_gradient_error(wl, sptr)
        out["errors_vs_oracle"] = ev
        out["cpu_baseline"] = {"value": ev["oracle_bead_steps"] / ev["oracle_seconds"],
                               "unit": "bead-steps/s (forward + gradient)", "cores": ev["oracle_threads"],
                               "kind": "oracle",
                               "sample": f"{ev['sample']}: the FP64 oracle's forward run with its pathwise "
                                         f"tangent in (rate, b, H), one thread a chain "
                                         f"({ev['oracle_seconds']:.1f} s wall)"}
    return out


def adjoint_gradient_error(wl, sptr, n_steps=2000, sample=(0, 255)):
    """The float32 adjoint's gradients against the FP64 oracle's pathwise
    tangent (same Philox draws, noise held fixed) on sampled chains of the
    differentiation workload, over its first n_steps steps (two checkpoint
    segments): max |difference| / max |gradient| per parameter (rate, b, H)."""
    import numpy as np
    import torch
    from oracle import oracle as O
    from paper_2206_05851_gb300 import bdra
    from paper_2206_05851_gb300 import inputs as I
    sample = [c for c in sample if c < len(wl.chains)]
    S = wl.window_steps
    W = n_steps // S
    pos0 = I.initial_positions(wl)
    offs = I.spring_offsets(wl.chains)
    G = np.zeros((W, int(offs[-1])))
    for c, ch in enumerate(wl.chains):
        G[:, offs[c] + (ch.n_beads - 1) // 2] = 1.0 / W
    gls = np.ones(len(wl.chains))
    ctx = bdra.Context(wl.chains, wl.dt, S, wl.seed, torch.from_numpy(pos0).cuda(),
                       precision=bdra.BD_PREC_FP32, max_windows=W, bell_mask=I.CRIT_RSF, stream=sptr,
                       checkpoint_steps=I.ADJOINT_CHECKPOINT_STEPS)
    ctx.step(n_steps)
    got = ctx.adjoint(G, gls)[sample]
    ctx.close()
    sub = [wl.chains[c] for c in sample]
    bo = I.bead_offsets(wl.chains)
    p0 = np.concatenate([pos0[bo[c]:bo[c + 1]] for c in sample])
    t = time.perf_counter()
    r, dr = O.rsf_tangent(sub, wl.dt, S, n_steps, wl.seed, p0, n_threads=len(sub), chain_ids=sample)
    t = time.perf_counter() - t
    so = I.spring_offsets(sub)
    want = np.zeros((len(sub), 3))
    for k, (c, ch) in enumerate(zip(sample, sub)):
        Gc = G[:, offs[c]:offs[c + 1]]
        seed = Gc - gls[c] * ch.k0 * ch.dx * np.exp(ch.dx * r[:, so[k]:so[k + 1]]) * S * wl.dt
        for j in range(3):
            want[k, j] = float((seed * dr[j][:, so[k]:so[k + 1]]).sum())
    err = np.abs(got - want).max(axis=0) / np.abs(want).max(axis=0)
    return {"sample": f"chains {sample}, first {n_steps} steps ({W} windows, "
                      f"{n_steps // I.ADJOINT_CHECKPOINT_STEPS} checkpoint segments)",
            "grad_max_rel_err": {"rate": float(err[0]), "b": float(err[1]), "H": float(err[2])},
            "oracle_seconds": t, "oracle_threads": len(sub),
            "oracle_bead_steps": sum(ch.n_replicas * ch.n_beads for ch in sub) * n_steps,
            "precision": "GPU float32 adjoint (FP64 reductions) vs the FP64 oracle's tangent"}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.only_rest:
        import torch
        from paper_2206_05851_gb300 import bdra, build as B
        if not B.up_to_date():
            B.build()
        bdra.load()
        print(json.dumps({"rest": rest_line(torch.cuda.current_stream().cuda_stream)}), flush=True)
        return
    if args.only_vwf:
        import torch
        from paper_2206_05851_gb300 import bdra, build as B
        if not B.up_to_date():
            B.build()
        bdra.load()
        print(json.dumps({"vwf": vwf_line(torch.cuda.current_stream().cuda_stream, args.chains)}),
              flush=True)
        return
    if args.only_hi:
        import torch
        from paper_2206_05851_gb300 import bdra, build as B
        if not B.up_to_date():
            B.build()
        bdra.load()
        print(json.dumps({"hi": hi_line(torch.cuda.current_stream().cuda_stream, args.chains,
                                         args.hi_steps)}), flush=True)
        return
    if args.only_collapsed:
        import torch
        from paper_2206_05851_gb300 import bdra, build as B
        if not B.up_to_date():
            B.build()
        bdra.load()
        print(json.dumps({"collapsed": collapsed_line(torch.cuda.current_stream().cuda_stream,
                                                      args.chains)}), flush=True)
        return
    if args.only_adjoint:
        import torch
        from paper_2206_05851_gb300 import bdra, build as B
        if not B.up_to_date():
            B.build()
        bdra.load()
        line = adjoint_line(torch.cuda.current_stream().cuda_stream, args.adjoint_chains,
                            args.adjoint_steps)
        print(json.dumps({"adjoint": line}), flush=True)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2206_05851_gb300 import bdra, build as B, shard
    from paper_2206_05851_gb300 import inputs as I

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 and not B.up_to_date():
        B.build()
    if world > 1:
        dist.barrier()
    bdra.load()
    sptr = torch.cuda.current_stream().cuda_stream
    issue_peak, issue_mixed, issue_fma = measured_issue_ceiling(sptr)   # outside any timed region
    philox_peak = bdra.bd_probe_philox_rounds(sptr)

    # one workload of world x the configuration's chains, split into contiguous
    # chain ranges (per-GPU work fixed as N grows: weak scaling)
    wl_all = make_workload(args, world)
    pos_all = I.initial_positions(wl_all)
    chains, pos0, base = shard.rank_share(wl_all.chains, pos_all, rank, world)
    wl = dataclasses.replace(wl_all, chains=chains)
    main_line, ctx = replica_line(wl, pos0, base, args.chunk, args.steps, args.warmup, sptr,
                                  args.autotune, issue_peak, philox_peak, dist if world > 1 else None,
                                  traffic_at=None if world > 1 else (BELL_TRAFFIC_AT if args.workload == "bell_16384"
                                                                     else REPLICA_TRAFFIC_AT),
                                  keep_ctx=True,
                                  lanes_hint=args.lanes_hint, layout_hint=args.layout_hint)
    out = {"metric": METRIC, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic"}
    out.update(main_line)
    out["config"]["parallelism"] = (
        f"one workload of {len(wl_all.chains)} chains split into {world} contiguous chain range(s) "
        f"balanced by N(R+1), global chain ids in the noise counter; no collective during the "
        f"integration; events and first-event arrays gathered after it")
    out["config"]["chains_total"] = len(wl_all.chains)
    # after the timed region: the whole workload's event list and kinetics on rank 0
    ev, _ = ctx.events(capacity=6 * ctx.M)
    events = shard.gather_events(shard.globalize_events(ev, base), dist if world > 1 else None)
    _, ft, fb = ctx.kinetics()
    ft_all = shard.gather_rows(ft, dist if world > 1 else None)
    fb_all = shard.gather_rows(fb, dist if world > 1 else None)
    if rank == 0:
        out["events_detected"] = int(len(events))
        if wl.thr_mask or wl.bell_mask:
            out["kinetics"] = kinetics_summary(ft_all, fb_all, wl_all.chains, wl.thr_mask, wl.bell_mask,
                                               args.chunk * args.steps, wl.dt)
    peaks = measured_peaks()
    if peaks:
        out["measured_peaks_file"] = {k: peaks[k] for k in list(peaks)[:8]}
    S = wl.window_steps
    chunk = args.chunk
    if rank == 0 and world == 1:
        value = out["value"]
        # plain FP64 path on the same chains, 1000 steps, and the FP32 force
        # error against it
        if not args.no_fp64:
            n64 = 1000
            c64 = bdra.Context(wl.chains, wl.dt, S, wl.seed, torch.from_numpy(pos0).cuda(),
                               precision=bdra.BD_PREC_FP64, max_windows=n64 // S + 1,
                               thr_mask=wl.thr_mask, bell_mask=wl.bell_mask, stream=sptr)
            c64.step(S)
            torch.cuda.synchronize()
            c64.set_positions(torch.from_numpy(pos0).cuda(), 0)
            torch.cuda.synchronize()
            stream = torch.cuda.current_stream()
            a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            c64.step(n64)
            b_.record(stream)
            torch.cuda.synchronize()
            t64 = a.elapsed_time(b_) / 1e3
            v64 = sum(c.n_replicas * c.n_beads for c in wl.chains) * n64 / t64
            ctx.set_positions(torch.from_numpy(pos0).cuda(), 0)
            ctx.step(n64)
            nw = n64 // S
            errs = []
            for w in range(nw):
                r32 = ctx.replica_average(w)
                r64 = c64.replica_average(w)
                errs.append(float(np.abs(r32 - r64).max() / np.abs(r64).max()))
            c64.close()
            out["fp64_plain"] = {"value": v64, "unit": "bead-steps/s",
                                 "sample": f"same {len(wl.chains)} chains, {n64} steps",
                                 "speedup_fp32_over_fp64": value / v64,
                                 "rsf_max_rel_err_fp32_vs_fp64": max(errs)}
        # end to end through the C ABI with host buffers
        if not args.no_e2e:
            bead_steps_chunk = wl.bead_steps(chunk)
            ev_cap = 6 * ctx.M
            pos_h = torch.from_numpy(pos0).pin_memory()
            ev_h = np.zeros(ev_cap, dtype=bdra.EVENT_DTYPE)
            rsf_h = np.zeros(ctx.M)
            e2e_steps = 2

            def e2e_step():
                bdra.bd_set_positions(ctx.ptr, pos_h, 0)
                ctx.step(chunk)
                n = bdra.bd_detect_events(ctx.ptr, ev_h, ev_cap, None)
                bdra.bd_replica_average(ctx.ptr, chunk // S - 1, rsf_h)
                return n

            e2e_step()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            nev = 0
            for _ in range(e2e_steps):
                nev = e2e_step()
            torch.cuda.synchronize()
            te = (time.perf_counter() - t0) / e2e_steps
            out["e2e"] = {"value": bead_steps_chunk / te, "unit": "bead-steps/s",
                          "h2d_bytes_per_step": int(pos_h.numel() * 8),
                          "d2h_bytes_per_step": int(nev * 24 + ctx.M * 8 + 8),
                          "steps": e2e_steps}
        ctx.close()
        if not args.no_adjoint:
            out["adjoint"] = adjoint_line(sptr, args.adjoint_chains, args.adjoint_steps,
                                          grad_check=not args.no_cpu)
        if not args.no_conformation:
            out["conformation"] = conformation_line(wl, pos0, sptr)
        # measured per-unit ceilings of this GPU (context for every fraction above)
        out["measured_unit_peaks"] = {
            "issue_lane_instr_per_s": issue_peak,
            "issue_mixed_fp32_int_lane_instr_per_s": issue_mixed,
            "issue_fp32_fma_lane_instr_per_s": issue_fma,
            "int_alu_lop3_per_s": bdra.bd_probe_int_alu(sptr),
            "philox_rounds_per_s": philox_peak,
            "fp32_fma_flops": bdra.bd_probe_fp32_fma(sptr),
            "fp64_fma_flops": bdra.bd_probe_fp64_fma(sptr),
            "mufu_rsqrt_per_s": bdra.bd_probe_mufu(sptr),
            "basis": "independent chains at full occupancy, no memory traffic (bd_probe_*)"}
        if not args.no_cpu:
            n_cpu = 20_000                               # about 10 s on 16 cores
            cpu, r, sample, sub_pos = cpu_baseline(wl, pos0, n_steps=n_cpu, keep=True)
            out["cpu_baseline"] = cpu
            out["errors_vs_oracle"] = errors_vs_oracle(wl, r, sample, sub_pos, n_cpu, sptr)
        if not args.no_batched:
            out["uneven"] = batch_line("uneven_4096", sptr, issue_peak, philox_peak, args)
            out["bell"] = batch_line("bell_16384", sptr, issue_peak, philox_peak, args)
        if not args.no_collapsed:
            out["collapsed"] = collapsed_line(sptr, issue_peak=issue_peak)
        if not args.no_hi:
            out["hi"] = hi_line(sptr)
        if not args.no_vwf:
            out["vwf"] = vwf_line(sptr)
    else:
        ctx.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()

if __name__ == "__main__":
    main()
