"""GPU parity for chains with hydrodynamic interaction (Eqs. 1-3): the
Rotne-Prager-Yamakawa diffusion tensor, its Cholesky factor for the
correlated noise and the mobility-weighted drift, one CTA per slot, against
the FP64 oracle on the same seeded inputs and Philox draws.

- Positions of parents and replicas, RSF and TSF profiles (per chain and
  window) within 1e-10 (FP64) / 1e-4 (FP32) relative; FP64 first-event steps
  equal; FP32 first-event steps equal except at near-ties, each checked
  against the oracle's own force or hazard at its step (parity_events.py).
- The paper's collapsed chain (N = 50, harmonic springs, Lennard-Jones, bead
  radius a = 1) in shear, smaller collapsed chains, FENE and Hookean chains
  with a bead radius in their own length unit, the two-bead chain, the
  largest chain (N = 64, tensor of 192 rows: 48 tile rows, five tiles on some
  threads), and free-draining chains in the same batch.
- Identical noise: every replica equals its parent (same kernel, same
  arithmetic).
"""
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


def _collapsed(N, R, flow=I.FLOW_SHEAR, rate=7.5, hi=1.0):
    return I.Chain(n_beads=N, n_replicas=R, spring=I.SPRING_HARMONIC, flow=flow, rate=rate,
                   H=400.0, r0=2.0, lj_u=1.0, lj_sigma=2.0, f_c=30.0, k0=50.0, dx=0.1, hi_a=hi)


def _collapsed_set():
    return [_collapsed(50, 3), _collapsed(12, 4, I.FLOW_NONE, 0.0), _collapsed(3, 2, I.FLOW_UNIAXIAL, 2.0),
            _collapsed(12, 3, hi=0.0)]                       # free draining in the same batch


def _fene_set():
    # thresholds and Bell rates set so that both kinds of event occur within
    # the 300 steps
    return [I.Chain(n_beads=20, n_replicas=3, spring=I.SPRING_FENE, flow=I.FLOW_UNIAXIAL, b=50.0,
                    rate=0.5, f_c=3.0, k0=1.0, dx=0.2, hi_a=0.5),
            I.Chain(n_beads=64, n_replicas=2, spring=I.SPRING_FENE, flow=I.FLOW_SHEAR, b=100.0,
                    rate=0.2, f_c=3.0, k0=1.0, dx=0.2, hi_a=0.4),
            I.Chain(n_beads=2, n_replicas=2, spring=I.SPRING_HOOKE, flow=I.FLOW_PLANAR, rate=0.3,
                    f_c=2.0, k0=1.0, dx=0.5, hi_a=0.3),
            I.Chain(n_beads=20, n_replicas=4, spring=I.SPRING_FENE, flow=I.FLOW_UNIAXIAL, b=50.0,
                    rate=0.5, f_c=3.0, k0=1.0, dx=0.2)]


def _tc_shapes_set():
    # the float32 tensor-core kernel's shapes besides 50 beads: the smallest
    # head (43 beads: 3 head rows, one 8-deep head update), no head with a
    # full 126-row trailing block (42), a partial last panel (33 beads: 99
    # rows) and a 15-row head (47)
    return [_collapsed(43, 2), _collapsed(42, 2, I.FLOW_NONE, 0.0), _collapsed(33, 2),
            _collapsed(47, 2, I.FLOW_UNIAXIAL, 2.0)]


SETS = {"collapsed": (_collapsed_set, 4e-5, 50, [20, 130, 150]),
        "fene": (_fene_set, 1e-3, 50, [20, 130, 150]),
        "tc_shapes": (_tc_shapes_set, 4e-5, 50, [20, 130, 150])}


def _gpu(chains, dt, S, steps, pos0, prec, seed=9, flags=0, thr=7, bell=7):
    import torch
    total = sum(steps)
    ctx = bdra.Context(chains, dt, S, seed, pos0, precision=prec, max_windows=total // S + 1,
                       thr_mask=thr, bell_mask=bell, flags=flags,
                       stream=torch.cuda.current_stream().cuda_stream)
    for n in steps:
        ctx.step(n)
    nw = total // S
    out = dict(pos=ctx.positions(False), allpos=ctx.positions(True),
               rsf=np.array([ctx.replica_average(w) for w in range(nw)]).reshape(nw, ctx.M),
               tsf=np.array([ctx.time_average(w) for w in range(nw)]).reshape(nw, ctx.M))
    out["haz"], out["first_thr"], out["first_bell"] = ctx.kinetics()
    out["info"] = ctx.info()
    ctx.close()
    return out


def _split(allpos, chains):
    par, rep, o = [], [], 0
    for c in chains:
        blk = allpos[o:o + (c.n_replicas + 1) * c.n_beads].reshape(c.n_replicas + 1, c.n_beads, 3)
        par.append(blk[0])
        rep.append(blk[1:].reshape(-1, 3))
        o += (c.n_replicas + 1) * c.n_beads
    return np.concatenate(par), np.concatenate(rep)


def _rel(got, want, sizes):
    worst, o = 0.0, 0
    for n in sizes:
        g, w = got[o:o + n], want[o:o + n]
        worst = max(worst, float(np.abs(g - w).max() / max(np.abs(w).max(), 1e-300)))
        o += n
    return worst


@pytest.fixture(scope="module", params=sorted(SETS))
def case(request):
    make, dt, S, steps = SETS[request.param]
    chains = make()
    pos0 = I.initial_positions(I.custom(chains, dt, S, sum(steps)), seed=29)
    r = O.run(chains, dt, S, sum(steps), 9, pos0, thr_mask=7, bell_mask=7, n_threads=8)
    return request.param, chains, dt, S, steps, pos0, r


@pytest.mark.parametrize("prec", PRECS)
def test_hi_chains_match_oracle(case, prec):
    name, chains, dt, S, steps, pos0, r = case
    g = _gpu(chains, dt, S, steps, pos0, prec)
    tol = TOL[prec]
    nb = [c.n_beads for c in chains]
    assert np.isfinite(g["allpos"]).all()
    assert _rel(g["pos"], O.com_frame(r["pos"], nb), nb) <= tol
    par, rep = _split(g["allpos"], chains)
    np.testing.assert_array_equal(par, g["pos"])
    sizes = [c.n_beads for c in chains for _ in range(c.n_replicas)]
    assert _rel(rep, O.com_frame(r["rep"], sizes), sizes) <= tol
    PE.check_profiles(g, r, chains, tol)
    assert (r["first_thr"] >= 0).sum() > 0 and (r["first_bell"] >= 0).sum() > 0
    if prec == bdra.BD_PREC_FP64:
        np.testing.assert_array_equal(g["first_thr"], r["first_thr"])
        np.testing.assert_array_equal(g["first_bell"], r["first_bell"])
        np.testing.assert_allclose(g["haz"], r["lam"], rtol=1e-9, atol=1e-300)
        assert g["info"].overextensions == int(r["overext"].sum())
    else:
        # float32: event steps exact up to near-ties; Bell hazards in log
        # space (a relative force error e moves k0 exp(dx f) by about dx f e)
        replay = PE.OracleReplay(chains, dt, S, 9, pos0, 7, 7)
        PE.compare_events_fp32(g, r, chains, S, replay)
        PE.compare_hazards_fp32(g["haz"], r["lam"])


def test_hi_moves_differently_from_free_draining():
    # the same chain and noise with and without the interaction part
    ch = _collapsed(12, 2)
    fd = _collapsed(12, 2, hi=0.0)
    pos0 = I.initial_positions(I.custom([ch], 4e-5, 50, 200), seed=3)
    a = _gpu([ch], 4e-5, 50, [200], pos0, bdra.BD_PREC_FP64, thr=0, bell=0)["pos"]
    b = _gpu([fd], 4e-5, 50, [200], pos0, bdra.BD_PREC_FP64, thr=0, bell=0)["pos"]
    assert np.abs(a - b).max() > 1e-3


@pytest.mark.parametrize("prec", PRECS)
def test_identical_noise_replicas_equal_parent(prec):
    chains = _collapsed_set()[:3]
    pos0 = I.initial_positions(I.custom(chains, 4e-5, 50, 120), seed=4)
    g = _gpu(chains, 4e-5, 50, [120], pos0, prec, flags=bdra.BD_FLAG_IDENTICAL_NOISE, thr=0, bell=0)
    par, rep = _split(g["allpos"], chains)
    o = po = 0
    for ch in chains:
        p = par[po:po + ch.n_beads]
        for k in range(ch.n_replicas):
            np.testing.assert_array_equal(rep[o + k * ch.n_beads:o + (k + 1) * ch.n_beads], p)
        o += ch.n_replicas * ch.n_beads
        po += ch.n_beads


@pytest.mark.parametrize("prec", [bdra.BD_PREC_FP64, bdra.BD_PREC_FP32])
def test_conformation_diagnostics_with_hi(prec):
    # Eq. 5 for the paper's set-up (collapsed chains with hydrodynamic
    # interaction in shear): D-bar per replica, per-bead D over replicas, R_GZ
    import torch
    chains = [_collapsed(50, 4), _collapsed(12, 3, I.FLOW_NONE, 0.0), _collapsed(12, 2, hi=0.0)]
    dt, S, n = 4e-5, 50, 150
    pos0 = I.initial_positions(I.custom(chains, dt, S, n), seed=17)
    ctx = bdra.Context(chains, dt, S, 9, pos0, precision=prec, max_windows=n // S,
                       flags=bdra.BD_FLAG_CONFORMATION, stream=torch.cuda.current_stream().cuda_stream)
    ctx.step(70)
    ctx.step(80)
    got = [ctx.conformation(w) for w in range(n // S)]
    ctx.close()
    want = O.conformation(chains, dt, S, n, 9, pos0)
    for k in range(3):
        g = np.array([x[k] for x in got])
        assert np.abs(g - want[k]).max() <= TOL[prec] * np.abs(want[k]).max(), k


def test_windows_across_chunks():
    # 75 windows of 2 steps: the step graph runs chunks of at most 64 windows,
    # so window snapshots and partial rows cross a chunk boundary (ring rows)
    chains = [_collapsed(12, 3), _collapsed(12, 2, hi=0.0),
              I.Chain(n_beads=9, n_replicas=3, spring=I.SPRING_FENE, flow=I.FLOW_SHEAR, b=50.0, rate=1.0,
                      hi_a=0.5)]
    dt, S, steps = 4e-5, 2, [61, 89]
    pos0 = I.initial_positions(I.custom(chains, dt, S, sum(steps)), seed=21)
    g = _gpu(chains, dt, S, steps, pos0, bdra.BD_PREC_FP64, thr=0, bell=0)
    r = O.run(chains, dt, S, sum(steps), 9, pos0, thr_mask=0, bell_mask=0, n_threads=4)
    assert g["rsf"].shape[0] == 75
    for key in ("rsf", "tsf"):
        assert np.abs(g[key] - r[key]).max() <= 1e-10 * np.abs(r[key]).max(), key
    nb = [c.n_beads for c in chains]
    assert _rel(g["pos"], O.com_frame(r["pos"], nb), nb) <= 1e-10


@pytest.mark.slow
def test_paper_rsf_spread_at_rest():
    # The paper's collapsed chain with RPY at rest (Sec. III, Fig. 2 set-up,
    # S = 0.02 tau): the spread of the middle (25th) spring's RSF over chains
    # and windows is 6.7 for N_R = 10 and 3.3 for N_R = 50. The same set-up
    # here (128 chains from the starting globules, windows 3-6) lands within
    # 15% of both, and the spread falls as N_R^-1/2 between them; the TSF
    # matches them (within 15%) at the sampling times the paper gives.
    import torch
    S, windows, skip = 2000, 6, 2
    spread = {}
    for R in (10, 50):
        chains = []
        for _ in range(128):
            ch = I.collapsed_chain(R, rate=0.0)
            ch.hi_a = 1.0
            chains.append(ch)
        pos0 = I.initial_positions(I.custom(chains, I.COLLAPSED_DT, S, windows * S), seed=12)
        ctx = bdra.Context(chains, I.COLLAPSED_DT, S, 12, pos0, precision=bdra.BD_PREC_FP32,
                           max_windows=windows, stream=torch.cuda.current_stream().cuda_stream)
        ctx.step(windows * S)
        rsf = np.array([ctx.replica_average(w) for w in range(skip, windows)])
        ctx.close()
        mid = I.spring_offsets(chains)[:-1] + 24
        spread[R] = rsf[:, mid].std()
    assert abs(spread[10] / 6.7 - 1) < 0.15 and abs(spread[50] / 3.3 - 1) < 0.15, spread
    assert abs(spread[10] / spread[50] / np.sqrt(5) - 1) < 0.15, spread
    # Fig. 2: the TSF reaches the same spread only with S = 0.07 tau (N_R = 10)
    # and S = 0.36 tau (N_R = 50)
    for s_tau, R in ((0.07, 10), (0.36, 50)):
        St = int(round(s_tau * 1e5))
        chains = []
        for _ in range(128):
            ch = I.collapsed_chain(1, rate=0.0)
            ch.hi_a = 1.0
            chains.append(ch)
        pos0 = I.initial_positions(I.custom(chains, I.COLLAPSED_DT, St, 3 * St), seed=12)
        ctx = bdra.Context(chains, I.COLLAPSED_DT, St, 12, pos0, precision=bdra.BD_PREC_FP32,
                           max_windows=3, stream=torch.cuda.current_stream().cuda_stream)
        ctx.step(3 * St)
        tsf = np.array([ctx.time_average(w) for w in (1, 2)])
        ctx.close()
        mid = I.spring_offsets(chains)[:-1] + 24
        assert abs(tsf[:, mid].std() / spread[R] - 1) < 0.15, (s_tau, tsf[:, mid].std(), spread)


@pytest.mark.slow
@pytest.mark.parametrize("hi", [0.0, 1.0])
def test_float32_trimer_samples_the_stationary_density(hi):
    # Long float32 runs of three collapsed beads at rest (kappa 50, u 2, rest
    # and sigma 2), free draining and with RPY: bond length and bead angle
    # against 3-D quadrature of exp(-U), as the oracle's pin, so that the
    # fast float path (approximate reciprocals and square roots, float32
    # Cholesky) is checked against the statics over 10^4 relaxation times of
    # a bond, not only against the oracle over short runs.
    import math
    import torch
    from scipy import integrate
    kappa, u, R0, SIG = 50.0, 2.0, 2.0, 2.0

    def weight(r1, r2, c):
        r02 = math.sqrt(max(r1 * r1 + r2 * r2 - 2 * r1 * r2 * c, 1e-12))
        x = SIG / r02
        return r1 * r1 * r2 * r2 * math.exp(-0.5 * kappa * ((r1 - R0) ** 2 + (r2 - R0) ** 2)
                                            - u * (x ** 12 - 2 * x ** 6))

    lo, hi_ = R0 - 1.0, R0 + 1.0
    opts = dict(epsabs=1e-13, epsrel=1e-8)
    Z = integrate.tplquad(lambda c, r2, r1: weight(r1, r2, c), lo, hi_, lo, hi_, -1, 1, **opts)[0]
    mc = integrate.tplquad(lambda c, r2, r1: c * weight(r1, r2, c), lo, hi_, lo, hi_, -1, 1, **opts)[0] / Z
    mr = integrate.tplquad(lambda c, r2, r1: r1 * weight(r1, r2, c), lo, hi_, lo, hi_, -1, 1, **opts)[0] / Z
    C, R, dt, steps = 512, 8, 2e-3, 40000
    chains = [I.Chain(n_beads=3, n_replicas=R, spring=I.SPRING_HARMONIC, H=kappa, r0=R0, lj_u=u,
                      lj_sigma=SIG, hi_a=hi) for _ in range(C)]
    pos0 = np.zeros((3 * C, 3))
    pos0[:, 2] = np.tile([0.0, 2.0, 4.0], C)
    ctx = bdra.Context(chains, dt, steps, 33, pos0, precision=bdra.BD_PREC_FP32, max_windows=1,
                       stream=torch.cuda.current_stream().cuda_stream)
    ctx.step(steps)
    allpos = ctx.positions(True).reshape(C, R + 1, 3, 3)
    ctx.close()
    q1, q2 = allpos[:, :, 1] - allpos[:, :, 0], allpos[:, :, 2] - allpos[:, :, 1]
    n1, n2 = np.linalg.norm(q1, axis=-1).ravel(), np.linalg.norm(q2, axis=-1).ravel()
    cos_bead = (-(q1 * q2).sum(axis=-1)).ravel() / (n1 * n2)
    for est, want in ((cos_bead, mc), (n1, mr)):
        sd = est.std() / math.sqrt(est.size)
        assert abs(est.mean() - want) < 5 * sd + 0.005 * abs(want), (est.mean(), want, sd)


def test_fene_floor_with_hi_matches_oracle_exactly():
    # FENE chains with RPY driven onto the FENE floor (strong uniaxial flow):
    # FP64 positions, floor counts and first events equal the oracle's
    chains = [I.Chain(n_beads=10, n_replicas=3, spring=I.SPRING_FENE, flow=I.FLOW_UNIAXIAL, b=20.0,
                      rate=4.0, f_c=3.0, k0=1e-3, dx=0.5, hi_a=0.5),
              I.Chain(n_beads=6, n_replicas=2, spring=I.SPRING_FENE, flow=I.FLOW_UNIAXIAL, b=20.0,
                      rate=8.0, f_c=3.0, k0=1e-3, dx=0.5, hi_a=0.5)]
    # 300 steps: long enough for the floor, short enough that the oracle's
    # laboratory-frame centre of mass (which grows as exp(rate t)) stays
    # small next to the chain, so its rounding stays below the tolerance
    dt, S, steps = 2e-3, 20, [130, 170]
    pos0 = I.initial_positions(I.custom(chains, dt, S, sum(steps)), seed=3)
    g = _gpu(chains, dt, S, steps, pos0, bdra.BD_PREC_FP64, seed=5)
    r = O.run(chains, dt, S, sum(steps), 5, pos0, thr_mask=7, bell_mask=7, n_threads=2)
    assert r["overext"].sum() > 10
    assert g["info"].overextensions == int(r["overext"].sum())
    nb = [c.n_beads for c in chains]
    assert _rel(g["pos"], O.com_frame(r["pos"], nb), nb) <= 1e-10
    np.testing.assert_array_equal(g["first_thr"], r["first_thr"])
    np.testing.assert_array_equal(g["first_bell"], r["first_bell"])
