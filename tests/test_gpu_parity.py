"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs and the same Philox draws.

Tolerances (relative, per chain, centre-of-mass frame; force profiles per
chain and window): 1e-10 in FP64 mode, 1e-4 in FP32 mode; event steps equal
in FP64 mode; FP32 event steps equal except at near-ties, checked one by one
against the oracle's own force or hazard at the earlier of the two steps
(parity_events.py: |f - f_c| < 1e-4 f_c; the Bell hazard within the float32
log-hazard tolerance of its Exp(1) level).
"""
import math

import numpy as np
import pytest

import parity_events as PE
from oracle import oracle as O
from paper_2206_05851_gb300 import bdra
from paper_2206_05851_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {bdra.BD_PREC_FP64: 1e-10, bdra.BD_PREC_FP32: 1e-4}
PRECS = [bdra.BD_PREC_FP64, bdra.BD_PREC_FP32]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2206_05851_gb300 import build as B
    B.build()
    torch.cuda.init()


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def gpu_run(chains, dt, S, steps, seed, pos0, prec, thr=7, bell=7, flags=0, lanes=0,
            want_all=True, layout=0):
    total = sum(steps)
    ctx = bdra.Context(chains, dt, S, seed, pos0, precision=prec, max_windows=total // S + 1,
                       thr_mask=thr, bell_mask=bell, flags=flags, stream=_stream(),
                       lanes_hint=lanes, layout_hint=layout)
    for n in steps:
        ctx.step(n)
    nw = total // S
    out = dict(pos=ctx.positions(False),
               allpos=ctx.positions(True) if want_all else None,
               rsf=np.array([ctx.replica_average(w) for w in range(nw)]).reshape(nw, ctx.M),
               tsf=np.array([ctx.time_average(w) for w in range(nw)]).reshape(nw, ctx.M))
    out["haz"], out["first_thr"], out["first_bell"] = ctx.kinetics()
    out["events"], out["log_surv"] = ctx.events()
    out["info"] = ctx.info()
    ctx.close()
    return out


def ora_run(chains, dt, S, n, seed, pos0, thr=7, bell=7, identical=False, chain_ids=None):
    return O.run(chains, dt, S, n, seed, pos0, thr_mask=thr, bell_mask=bell,
                 identical_noise=identical, n_threads=8, chain_ids=chain_ids)


def _split_replicas(allpos, chains):
    """GPU all-slot array -> (parents, replicas chain-major) like the oracle."""
    par, rep, o = [], [], 0
    for c in chains:
        blk = allpos[o:o + (c.n_replicas + 1) * c.n_beads].reshape(c.n_replicas + 1, c.n_beads, 3)
        par.append(blk[0])
        rep.append(blk[1:].reshape(-1, 3))
        o += (c.n_replicas + 1) * c.n_beads
    return np.concatenate(par), np.concatenate(rep)


def rel_err_chains(got, want, sizes):
    worst, o = 0.0, 0
    for n in sizes:
        g, w = got[o:o + n], want[o:o + n]
        worst = max(worst, float(np.abs(g - w).max() / max(np.abs(w).max(), 1e-300)))
        o += n
    return worst


def compare_states(g, r, chains, tol):
    nb = [c.n_beads for c in chains]
    assert rel_err_chains(g["pos"], O.com_frame(r["pos"], nb), nb) <= tol
    if g["allpos"] is not None:
        par, rep = _split_replicas(g["allpos"], chains)
        np.testing.assert_array_equal(par, g["pos"])
        sizes = [c.n_beads for c in chains for _ in range(c.n_replicas)]
        assert rel_err_chains(rep, O.com_frame(r["rep"], sizes), sizes) <= tol


def compare_profiles(g, r, chains, tol):
    PE.check_profiles(g, r, chains, tol)


def compare_events_exact(g, r):
    np.testing.assert_array_equal(g["first_thr"], r["first_thr"])
    np.testing.assert_array_equal(g["first_bell"], r["first_bell"])
    np.testing.assert_allclose(g["haz"], r["lam"], rtol=1e-9, atol=1e-300)


def compare_events_fp32(g, r, chains, dt, S, seed, pos0, thr=7, bell=7, chain_ids=None, cols=None):
    """Event steps equal the oracle's except at near-ties (each checked at its
    step against the oracle's own force or hazard); hazards in log space."""
    replay = PE.OracleReplay(chains, dt, S, seed, pos0, thr, bell, chain_ids)
    counts = PE.compare_events_fp32(g, r, chains, S, replay, cols=cols)
    PE.compare_hazards_fp32(g["haz"] if cols is None else g["haz"][:, cols], r["lam"])
    return counts


def c1_like(rate_wi=2.0, n=20, R=16, b=50.0):
    return I.Chain(n_beads=n, n_replicas=R, spring=I.SPRING_FENE, flow=I.FLOW_UNIAXIAL, H=1.0,
                   b=b, rate=I.rate_from_wi(rate_wi, n), f_c=0.9 * math.sqrt(b))


# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", PRECS)
def test_normals_match_oracle(prec):
    rng = np.random.default_rng(0)
    n = 200_000
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:, 1] &= 0x00FFFFFF
    seed = 0x1234_5678_9ABC_DEF0
    got = np.zeros((n, 3))
    bdra.bd_philox_normals(seed, ctr, prec, got)
    want = O.normals3_many(seed, ctr)
    if prec == bdra.BD_PREC_FP64:
        np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)
    else:
        err = np.abs(got - want)
        assert np.median(err) < 1e-6
        assert np.quantile(err, 0.999) < 2e-5
        assert err.max() < 2e-3       # rare draws with u -> 1 (tiny normal, coarse log)


@pytest.mark.parametrize("prec", PRECS)
def test_single_chain_1000_steps(prec):
    wl = I.single_chain_fp64(n_steps=1000)
    pos0 = I.initial_positions(wl)
    g = gpu_run(wl.chains, wl.dt, wl.window_steps, [1000], wl.seed, pos0, prec)
    r = ora_run(wl.chains, wl.dt, wl.window_steps, 1000, wl.seed, pos0)
    compare_states(g, r, wl.chains, TOL[prec])
    compare_profiles(g, r, wl.chains, TOL[prec])
    assert g["info"].overextensions == int(r["overext"].sum()) == 0


def _ragged_chains():
    spec = [(2, 1, I.FLOW_NONE, 0.0), (5, 3, I.FLOW_SHEAR, 1.5), (20, 16, I.FLOW_UNIAXIAL, 0.3),
            (33, 7, I.FLOW_PLANAR, 0.2), (100, 64, I.FLOW_PLANAR, 0.01),
            (129, 9, I.FLOW_SHEAR, 0.05), (257, 5, I.FLOW_UNIAXIAL, 0.002),
            (500, 130, I.FLOW_SHEAR, 0.01)]
    out = []
    for k, (n, R, flow, rate) in enumerate(spec):
        b = 20.0 + 15 * k
        out.append(I.Chain(n_beads=n, n_replicas=R, spring=I.SPRING_FENE, flow=flow, H=1.0 + 0.1 * k,
                           b=b, rate=rate, f_c=0.35 * math.sqrt(b * (1.0 + 0.1 * k)),
                           k0=1e-3, dx=1.0 / math.sqrt(b)))
    return out


@pytest.mark.parametrize("prec", PRECS)
def test_ragged_batch_split_calls(prec):
    chains = _ragged_chains()
    S, dt, seed = 7, 1e-3, 11
    steps = [10, 1, 33, 96]          # 140 steps = 20 windows; calls end mid-window
    pos0 = I.initial_positions(I.custom(chains, dt, S, 140), seed=5)
    g = gpu_run(chains, dt, S, steps, seed, pos0, prec)
    r = ora_run(chains, dt, S, 140, seed, pos0)
    compare_states(g, r, chains, TOL[prec])
    compare_profiles(g, r, chains, TOL[prec])
    if prec == bdra.BD_PREC_FP64:
        compare_events_exact(g, r)
    else:
        compare_events_fp32(g, r, chains, dt, S, seed, pos0)


def _event_chains(extreme: bool):
    """Event-rich chains. The extreme set drives springs onto the FENE floor
    (and Bell hazards to overflow): the FP64 path must still match the oracle
    exactly. The FP32 comparison uses the moderate set, which stays off the
    floor: float32 and float64 can take different floor decisions, after
    which the trajectories legitimately part."""
    b = 30.0
    r0, r1, fc, dx = (0.8, 3.0, 0.55, 8.0) if extreme else (0.25, 1.5, 0.4, 4.0)
    return [I.Chain(n_beads=16, n_replicas=24, spring=I.SPRING_FENE, flow=I.FLOW_UNIAXIAL,
                    b=b, rate=r0, f_c=fc * math.sqrt(b), k0=1e-4, dx=dx / math.sqrt(b)),
            I.Chain(n_beads=40, n_replicas=12, spring=I.SPRING_FENE, flow=I.FLOW_SHEAR,
                    b=b, rate=r1, f_c=fc * math.sqrt(b), k0=1e-4, dx=dx / math.sqrt(b)),
            I.Chain(n_beads=9, n_replicas=5, spring=I.SPRING_HOOKE, flow=I.FLOW_PLANAR,
                    b=b, rate=0.4, f_c=2.5, k0=1e-3, dx=1.0)]


@pytest.mark.parametrize("prec", PRECS)
def test_events_and_kinetics(prec):
    chains = _event_chains(extreme=prec == bdra.BD_PREC_FP64)
    S, dt, n, seed = 20, 2e-3, 2000, 3
    pos0 = I.initial_positions(I.custom(chains, dt, S, n), seed=8)
    g = gpu_run(chains, dt, S, [n], seed, pos0, prec, want_all=False)
    r = ora_run(chains, dt, S, n, seed, pos0)
    assert (r["first_thr"] >= 0).sum() > 20 and (r["first_bell"] >= 0).sum() > 10
    assert g["info"].overextensions == int(r["overext"].sum())
    if prec == bdra.BD_PREC_FP64:
        assert r["overext"].sum() > 0
        compare_events_exact(g, r)
    else:
        assert r["overext"].sum() == 0
        counts = compare_events_fp32(g, r, chains, dt, S, seed, pos0)
        assert counts["thr_equal"] > 20 and counts["bell_equal"] > 10, counts
    # the event list is the kinetic state, in (chain, spring, criterion, kind) order
    ev = g["events"]
    so = I.spring_offsets(chains)
    m = so[ev["chain"]] + ev["spring"]
    for e, mm in zip(ev, m):
        arr = g["first_thr"] if e["kind"] == 0 else g["first_bell"]
        assert arr[e["criterion"], mm] == e["step"]
    assert len(ev) == (g["first_thr"] >= 0).sum() + (g["first_bell"] >= 0).sum()
    keys = list(zip(ev["chain"], ev["spring"], ev["criterion"], ev["kind"]))
    assert keys == sorted(keys)
    # log-survival = -sum of hazards per chain and criterion
    for c in range(len(chains)):
        np.testing.assert_allclose(g["log_surv"][c], -g["haz"][:, so[c]:so[c + 1]].sum(axis=1),
                                   rtol=1e-12)


def test_fp32_isf_hazard_beyond_the_float32_range():
    # A float32 run sums each step's ISF Bell increment k0 dt e^(dx f) in a
    # float-float pair only while it lies within e^(+-64); larger ones (past
    # float32 range once summed) and smaller ones (lost in a float32 sum) go
    # to the float64 hazard directly. With k0 dt = 2e-40 and dx = 25 a
    # tension below 1.08 gives the small ones, above 6.2 the large ones (and
    # the events); hazards in log space and first passages as the oracle's,
    # off the FENE floor.
    b = 30.0
    chains = [I.Chain(n_beads=8, n_replicas=2, spring=I.SPRING_FENE, flow=I.FLOW_UNIAXIAL, b=b,
                      rate=0.3, f_c=1e9, k0=1e-37, dx=25.0),
              I.Chain(n_beads=12, n_replicas=3, spring=I.SPRING_FENE, flow=I.FLOW_SHEAR, b=b,
                      rate=1.0, f_c=1e9, k0=1e-37, dx=25.0)]
    S, dt, n, seed = 10, 2e-3, 1000, 5
    pos0 = I.initial_positions(I.custom(chains, dt, S, n), seed=3)
    g = gpu_run(chains, dt, S, [n], seed, pos0, bdra.BD_PREC_FP32, thr=0, bell=1, want_all=False)
    r = ora_run(chains, dt, S, n, seed, pos0, thr=0, bell=1)
    assert r["overext"].sum() == 0
    lam = r["lam"][0]
    big = math.exp(64.0)
    assert (lam > big).any() and (lam < big).any(), (lam.min(), lam.max())
    counts = compare_events_fp32(g, r, chains, dt, S, seed, pos0, thr=0, bell=1)
    assert counts["bell_equal"] >= 3, counts


@pytest.mark.parametrize("prec,layout", [(bdra.BD_PREC_FP64, 0), (bdra.BD_PREC_FP32, 1),
                                         (bdra.BD_PREC_FP32, 2)])
def test_identical_noise_replicas_reproduce_parent(prec, layout):
    # the parent kernel (one slot per lane) and the replica kernels (one or
    # two replicas per lane) round every step identically
    chains = _ragged_chains()[:6]
    S, dt = 13, 1e-3
    pos0 = I.initial_positions(I.custom(chains, dt, S, 91), seed=2)
    g = gpu_run(chains, dt, S, [91], 4, pos0, prec, flags=bdra.BD_FLAG_IDENTICAL_NOISE,
                layout=layout)
    par, rep = _split_replicas(g["allpos"], chains)
    o = 0
    for c, ch in enumerate(chains):
        p = g["pos"][sum(x.n_beads for x in chains[:c]):][:ch.n_beads]
        for k in range(ch.n_replicas):
            np.testing.assert_array_equal(rep[o + k * ch.n_beads:o + (k + 1) * ch.n_beads], p)
        o += ch.n_replicas * ch.n_beads


@pytest.mark.parametrize("prec", PRECS)
def test_results_do_not_depend_on_tile(prec):
    chains = [I.Chain(n_beads=31, n_replicas=11, spring=I.SPRING_FENE, flow=I.FLOW_SHEAR,
                      b=40.0, rate=1.0, f_c=3.0, k0=1e-3, dx=0.3),
              I.Chain(n_beads=20, n_replicas=40, spring=I.SPRING_FENE, flow=I.FLOW_UNIAXIAL,
                      b=40.0, rate=0.2, f_c=3.0, k0=1e-3, dx=0.3)]
    S, dt = 10, 1e-3
    pos0 = I.initial_positions(I.custom(chains, dt, S, 60), seed=9)
    if prec == bdra.BD_PREC_FP32:      # one and two replicas per lane (packed float32)
        shapes = [(1, L) for L in range(4, 17)] + [(2, L) for L in range(4, 8)]
    else:
        shapes = [(1, L) for L in (2, 4, 7, 10, 13, 16)]
    runs = [gpu_run(chains, dt, S, [60], 7, pos0, prec, lanes=L, layout=lay) for lay, L in shapes]
    for g in runs[1:]:
        # trajectories, parent samples and kinetics are bitwise the same
        for key in ("allpos", "tsf", "first_thr", "first_bell"):
            np.testing.assert_array_equal(g[key], runs[0][key])
        # the tile decides how replicas split into CTAs, hence the order of
        # the float64 replica sum: equal up to its last bits (exactly equal
        # in FP32 mode, where the float64 sums of float samples are exact)
        np.testing.assert_allclose(g["rsf"], runs[0]["rsf"], rtol=2e-15, atol=0)
        np.testing.assert_allclose(g["haz"], runs[0]["haz"], rtol=1e-14, atol=0)
        if prec == bdra.BD_PREC_FP32:
            np.testing.assert_array_equal(g["rsf"], runs[0]["rsf"])


@pytest.mark.parametrize("prec", PRECS)
def test_edge_cases(prec):
    # N = 2 (one spring), R = 1, window of one step
    ch = [I.Chain(n_beads=2, n_replicas=1, spring=I.SPRING_FENE, b=10.0, f_c=2.0, k0=1e-2, dx=0.5)]
    pos0 = np.array([[0.0, 0.0, 0.0], [1.0, 0.5, -0.2]])
    g = gpu_run(ch, 1e-3, 1, [5, 0, 7], 1, pos0, prec)
    r = ora_run(ch, 1e-3, 1, 12, 1, pos0)
    compare_states(g, r, ch, TOL[prec])
    compare_profiles(g, r, ch, TOL[prec])
    # maximum chain length (512 beads, 16 springs per lane, 32 lanes per slot)
    ch = [I.Chain(n_beads=512, n_replicas=3, spring=I.SPRING_FENE, flow=I.FLOW_SHEAR, b=100.0,
                  rate=0.01)]
    pos0 = I.initial_positions(I.custom(ch, 1e-3, 4, 12), seed=3)
    g = gpu_run(ch, 1e-3, 4, [12], 2, pos0, prec, thr=0, bell=0)
    r = ora_run(ch, 1e-3, 4, 12, 2, pos0, thr=0, bell=0)
    compare_states(g, r, ch, TOL[prec])
    compare_profiles(g, r, ch, TOL[prec])


@pytest.mark.parametrize("R", [1000, 4096])
def test_many_replica_groups(R):
    # 1000 replicas and the maximum 4096 of a short chain: many work items per
    # chain, one parent copy
    ch = [I.Chain(n_beads=24, n_replicas=R, spring=I.SPRING_FENE, flow=I.FLOW_PLANAR,
                  b=50.0, rate=0.05)]
    pos0 = I.initial_positions(I.custom(ch, 1e-3, 10, 30), seed=4)
    for prec in PRECS:
        g = gpu_run(ch, 1e-3, 10, [30], 6, pos0, prec, thr=0, bell=0)
        r = ora_run(ch, 1e-3, 10, 30, 6, pos0, thr=0, bell=0)
        compare_states(g, r, ch, TOL[prec])
        compare_profiles(g, r, ch, TOL[prec])


def test_capacity_and_state_errors():
    ch = [I.Chain(n_beads=8, n_replicas=2, spring=I.SPRING_FENE, b=20.0, f_c=0.1)]
    pos0 = I.initial_positions(I.custom(ch, 1e-3, 5, 10), seed=1)
    ctx = bdra.Context(ch, 1e-3, 5, 0, pos0, max_windows=2, thr_mask=7, stream=_stream())
    ctx.step(10)
    with pytest.raises(bdra.BdError) as e:
        ctx.step(5)
    assert e.value.status == bdra.BD_E_CAPACITY
    with pytest.raises(bdra.BdError):
        ctx.replica_average(2)
    # event capacity: count still reported
    out = np.zeros(1, dtype=bdra.EVENT_DTYPE)
    with pytest.raises(bdra.BdError) as e:
        bdra.bd_detect_events(ctx.ptr, out, 1)
    assert e.value.status == bdra.BD_E_CAPACITY
    with pytest.raises(bdra.BdError):
        ctx.set_positions(pos0, step=3)
    ctx.close()


def test_restart_and_spawn():
    chains = _ragged_chains()[1:4]
    S, dt = 10, 1e-3
    pos0 = I.initial_positions(I.custom(chains, dt, S, 40), seed=6)
    ctx = bdra.Context(chains, dt, S, 3, pos0, precision=bdra.BD_PREC_FP64, max_windows=8,
                       thr_mask=7, bell_mask=7, stream=_stream())
    ctx.step(25)
    ctx.set_positions(pos0, 0)          # restart from the same conformation
    ctx.step(40)
    again = ctx.positions(True)
    fresh = gpu_run(chains, dt, S, [40], 3, pos0, bdra.BD_PREC_FP64)
    np.testing.assert_array_equal(again, fresh["allpos"])
    np.testing.assert_array_equal(ctx.kinetics()[1], fresh["first_thr"])
    ctx.step(5)
    ctx.spawn()
    par, rep = _split_replicas(ctx.positions(True), chains)
    o, po = 0, 0
    for ch in chains:
        for k in range(ch.n_replicas):
            np.testing.assert_allclose(rep[o + k * ch.n_beads:o + (k + 1) * ch.n_beads],
                                       par[po:po + ch.n_beads], rtol=0, atol=1e-12)
        o += ch.n_replicas * ch.n_beads
        po += ch.n_beads
    ctx.close()


def test_device_and_host_buffers_agree():
    import torch
    chains = _ragged_chains()[2:4]
    pos0 = I.initial_positions(I.custom(chains, 1e-3, 10, 30), seed=1)
    ctx = bdra.Context(chains, 1e-3, 10, 2, torch.from_numpy(pos0).cuda(), max_windows=3,
                       thr_mask=7, stream=_stream())
    ctx.step(30)
    d = torch.zeros(ctx.M, dtype=torch.float64, device="cuda")
    bdra.bd_replica_average(ctx.ptr, 2, d)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(d.cpu().numpy(), ctx.replica_average(2))
    ctx.close()


def test_tsf_is_the_float64_mean_of_the_float32_isf_samples():
    # TSF (Sec. II) of a float32 run: the mean over the S = 1500 steps of a
    # window of the parent's float32 ISF samples, summed in a float-float
    # pair (error-free TwoSum, renormalised). The parent's trajectory does
    # not depend on the window length (its noise is keyed by the global
    # step), so a second run with one-step windows returns each ISF sample
    # itself as its TSF; their float64 means must equal the S = 1500 run's
    # TSF within the pair's bound, S 2^-47 of the mean |sample| (a plain
    # float32 sum of 1500 samples is off by about 3e-7 of their size). FENE
    # springs under strong elongation, and the free-draining collapsed and
    # vWF chains (signed forces, Lennard-Jones cohesion).
    fene = I.Chain(n_beads=16, n_replicas=1, spring=I.SPRING_FENE, flow=I.FLOW_UNIAXIAL, b=100.0,
                   rate=10.0)
    chains = [fene, I.collapsed_chain(1), I.vwf_chain(1, n_beads=20, hi=False)]
    dt, S, n = I.COLLAPSED_DT, 1500, 3000
    pos0 = I.initial_positions(I.custom(chains, dt, S, n), seed=12)
    runs = []
    for s in (S, 1):
        ctx = bdra.Context(chains, dt, s, 3, pos0, precision=bdra.BD_PREC_FP32,
                           max_windows=n // s, thr_mask=0, bell_mask=0, stream=_stream())
        ctx.step(n)
        runs.append((ctx.positions(False), np.array([ctx.time_average(w) for w in range(n // s)])))
        ctx.close()
    np.testing.assert_array_equal(runs[0][0], runs[1][0])
    isf = runs[1][1].reshape(n // S, S, -1)
    want = isf.mean(axis=1)
    scale = np.abs(isf).mean(axis=1)
    err = np.abs(runs[0][1] - want) / scale
    assert err.max() <= S * 2.0 ** -47, err.max()


def _sampled(wl, g, pos0, sample, n):
    """Sampled chains of a full-size float32 run against the oracle, which
    re-runs them alone with their global chain ids in the noise counter:
    positions per chain, RSF / TSF per (chain, window), Bell hazards in log
    space, and every event step equal up to the near-ties the oracle's own
    forces and hazards show."""
    boff, soff = I.bead_offsets(wl.chains), I.spring_offsets(wl.chains)
    sub = [wl.chains[c] for c in sample]
    sub_pos = np.concatenate([pos0[boff[c]:boff[c + 1]] for c in sample])
    r = ora_run(sub, wl.dt, wl.window_steps, n, wl.seed, sub_pos, thr=wl.thr_mask,
                bell=wl.bell_mask, chain_ids=sample)
    nb = [c.n_beads for c in sub]
    got = np.concatenate([g["pos"][boff[c]:boff[c + 1]] for c in sample])
    assert rel_err_chains(got, O.com_frame(r["pos"], nb), nb) <= 1e-4
    cols = np.concatenate([np.arange(soff[c], soff[c + 1]) for c in sample])
    PE.check_profiles({k: g[k][:, cols] for k in ("rsf", "tsf")}, r, sub, 1e-4)
    counts = compare_events_fp32(g, r, sub, wl.dt, wl.window_steps, wl.seed, sub_pos,
                                 wl.thr_mask, wl.bell_mask, chain_ids=sample, cols=cols)
    return r, counts


def _full_size(wl, n, autotune=False):
    ctx = bdra.Context(wl.chains, wl.dt, wl.window_steps, wl.seed, I.initial_positions(wl),
                       precision=bdra.BD_PREC_FP32, max_windows=n // wl.window_steps + 1,
                       thr_mask=wl.thr_mask, bell_mask=wl.bell_mask, stream=_stream())
    if autotune:
        ctx.autotune(probe_steps=8)
    ctx.step(n)
    nw = n // wl.window_steps
    g = dict(pos=ctx.positions(False),
             rsf=np.array([ctx.replica_average(w) for w in range(nw)]).reshape(nw, ctx.M),
             tsf=np.array([ctx.time_average(w) for w in range(nw)]).reshape(nw, ctx.M))
    g["haz"], g["first_thr"], g["first_bell"] = ctx.kinetics()
    ctx.close()
    return g


def test_full_size_sampled_parity():
    # The benchmark's launch configuration: 1024 chains, N = 100, 64 replicas,
    # planar elongation Wi = 5, FP32 integration, 1000 steps. Sampled chains
    # are re-run on their own by the oracle (same chain ids in the noise
    # counter).
    wl = I.planar_1024(n_steps=1000)
    g = _full_size(wl, 1000)
    _sampled(wl, g, I.initial_positions(wl), [0, 517, 1023], 1000)


def test_full_size_uneven_batch_sampled_parity():
    # C3 launch configuration: 4096 chains of 20..500 beads and 8..128
    # replicas, shear and elongation, one persistent launch per step variant,
    # shapes picked by the autotuner; FP32, 1000 steps; sampled chains of
    # different shapes re-run alone by the oracle
    wl = I.uneven_4096(n_steps=1000)
    g = _full_size(wl, 1000, autotune=True)
    sizes = [(c.n_beads, c.n_replicas) for c in wl.chains]
    sample = [int(np.argmax([n for n, _ in sizes])), int(np.argmin([n for n, _ in sizes])),
              int(np.argmax([r for _, r in sizes])), 1234, 4095]
    _sampled(wl, g, I.initial_positions(wl), sample, 1000)


def test_full_size_bell_workload_sampled_parity():
    # C4 launch configuration: 16384 chains, N = 50, 32 replicas, start-up
    # uniaxial Wi = 10, Bell and threshold criteria on ISF, TSF and RSF; FP32,
    # 1000 steps; sampled chains against the oracle
    wl = I.bell_16384(n_steps=1000)
    g = _full_size(wl, 1000)
    _sampled(wl, g, I.initial_positions(wl), [0, 8191, 16383], 1000)


@pytest.mark.parametrize("prec", PRECS)
def test_autotune_changes_shapes_not_results(prec):
    # the autotuner times every step variant and re-plans; results must not move
    chains = _ragged_chains()
    S, dt, seed, n = 7, 1e-3, 11, 70
    pos0 = I.initial_positions(I.custom(chains, dt, S, n), seed=5)
    base = gpu_run(chains, dt, S, [n], seed, pos0, prec)
    ctx = bdra.Context(chains, dt, S, seed, pos0, precision=prec, max_windows=n // S + 1,
                       thr_mask=7, bell_mask=7, stream=_stream())
    ctx.autotune(probe_steps=8, force=True)
    variants, groups, costs = ctx.plan()
    assert all(c > 0 for c in costs.values())
    for ch, v, g in zip(chains, variants, groups):
        L = v % 100
        per_warp = (2 if v >= 100 else 1) * (32 // -(-ch.n_beads // L))
        R = ch.n_replicas
        if v >= 100 or per_warp == 1:
            want = -(-R // per_warp)
        else:        # odd and even replicas in separate items (one noise half a warp)
            want = -(-((R + 1) // 2) // per_warp) + -(-(R // 2) // per_warp)
        assert -(-ch.n_beads // L) <= 32 and g == want
    ctx.step(n)
    allpos = ctx.positions(True)
    rsf = np.array([ctx.replica_average(w) for w in range(n // S)])
    with pytest.raises(bdra.BdError) as e:       # only before the first step
        ctx.autotune(8)
    assert e.value.status == bdra.BD_E_STATE
    ctx.close()
    np.testing.assert_array_equal(allpos, base["allpos"])
    if prec == bdra.BD_PREC_FP32:
        np.testing.assert_array_equal(rsf, base["rsf"])
    else:
        np.testing.assert_allclose(rsf, base["rsf"], rtol=2e-15, atol=0)
