"""GPU parity for the coarse-grained vWF chain (supplementary material, Table
S1, in the library's units): A2 domains (FENE in parallel with harmonic) on
the even springs, disulfide bonds on the odd springs, Lennard-Jones
cohesion, with and without RPY hydrodynamic interaction, against the FP64
oracle on the same seeded inputs and Philox draws.

- Positions of parents and replicas, RSF and TSF (per chain and window)
  within 1e-10 (FP64) / 1e-4 (FP32) relative; FP64 first-event steps and
  hazards equal (a raised unfolding rate, so that A2 domains unfold within
  the run); FP32 first-event steps equal except at near-ties checked against
  the oracle's own force or hazard at their step.
- Disulfide bonds never have events and keep a zero hazard.
- Chains of 50 beads (the paper's), an odd bead count (a last A2 domain
  without a following bond), 7 beads with hydrodynamic interaction, and the
  two-bead chain (one A2 domain).
"""
import numpy as np
import pytest

import parity_events as PE
from oracle import oracle as O
from paper_2206_05851_gb300 import bdra
from paper_2206_05851_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {bdra.BD_PREC_FP64: 1e-10, bdra.BD_PREC_FP32: 1e-4}
DT, S, STEPS = 4e-5, 50, [30, 170, 100]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2206_05851_gb300 import build as B
    B.build()
    torch.cuda.init()


def _chain(N, R, hi):
    c = I.vwf_chain(R, n_beads=N, hi=hi)
    c.k0 = 0.5            # raised so that A2 domains unfold within 300 steps
    c.f_c = 25.0
    return c


def _chains():
    return [_chain(50, 6, False), _chain(50, 3, True), _chain(11, 4, False), _chain(7, 3, True),
            _chain(2, 2, False)]


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


@pytest.fixture(scope="module")
def oracle_run():
    chains = _chains()
    pos0 = I.initial_positions(I.custom(chains, DT, S, sum(STEPS)), seed=31)
    r = O.run(chains, DT, S, sum(STEPS), 5, pos0, thr_mask=7, bell_mask=7, n_threads=8)
    return chains, pos0, r


@pytest.mark.parametrize("prec", [bdra.BD_PREC_FP64, bdra.BD_PREC_FP32])
def test_vwf_chains_match_oracle(oracle_run, prec):
    import torch
    chains, pos0, r = oracle_run
    ctx = bdra.Context(chains, DT, S, 5, pos0, precision=prec, max_windows=sum(STEPS) // S + 1,
                       thr_mask=7, bell_mask=7, stream=torch.cuda.current_stream().cuda_stream)
    for n in STEPS:
        ctx.step(n)
    nw = sum(STEPS) // S
    pos, allpos = ctx.positions(False), ctx.positions(True)
    rsf = np.array([ctx.replica_average(w) for w in range(nw)])
    tsf = np.array([ctx.time_average(w) for w in range(nw)])
    haz, first_thr, first_bell = ctx.kinetics()
    ctx.close()
    tol = TOL[prec]
    nb = [c.n_beads for c in chains]
    assert _rel(pos, O.com_frame(r["pos"], nb), nb) <= tol
    par, rep = _split(allpos, chains)
    sizes = [c.n_beads for c in chains for _ in range(c.n_replicas)]
    assert _rel(rep, O.com_frame(r["rep"], sizes), sizes) <= tol
    PE.check_profiles(dict(rsf=rsf, tsf=tsf), r, chains, tol)
    offs = I.spring_offsets(chains)
    odd = np.concatenate([np.arange(offs[c] + 1, offs[c + 1], 2) for c in range(len(chains))])
    assert (first_thr[:, odd] < 0).all() and (first_bell[:, odd] < 0).all() and (haz[:, odd] == 0).all()
    assert (r["first_bell"] >= 0).sum() >= 5 and (r["first_thr"] >= 0).sum() >= 5
    if prec == bdra.BD_PREC_FP64:
        np.testing.assert_array_equal(first_thr, r["first_thr"])
        np.testing.assert_array_equal(first_bell, r["first_bell"])
        np.testing.assert_allclose(haz, r["lam"], rtol=1e-9, atol=1e-300)
    else:
        # float32: event steps exact up to near-ties; hazards in log space (a
        # relative force error e moves k0 exp(dx f) by about dx f e)
        g = dict(first_thr=first_thr, first_bell=first_bell)
        PE.compare_events_fp32(g, r, chains, S, PE.OracleReplay(chains, DT, S, 5, pos0, 7, 7))
        PE.compare_hazards_fp32(haz, r["lam"])


@pytest.mark.slow
def test_float32_vwf_trimer_samples_the_stationary_density():
    # one A2 domain (FENE in parallel with harmonic) and one disulfide bond,
    # Lennard-Jones between the ends, at rest, float32 with RPY: both bond
    # lengths and the bead angle against 3-D quadrature of exp(-U)
    import math
    import torch
    from scipy import integrate
    fa, fb, xmax, H, u, R0, SIG = 20.0, 30.0, 0.8, 50.0, 2.0, 2.0, 2.0

    def weight(r1, r2, c):
        x1, x2 = r1 - R0, r2 - R0
        if abs(x1) >= xmax:
            return 0.0
        ua2 = 0.5 * fb * x1 * x1 - 0.5 * fa * xmax ** 2 * math.log(1 - (x1 / xmax) ** 2)
        r02 = math.sqrt(max(r1 * r1 + r2 * r2 - 2 * r1 * r2 * c, 1e-12))
        s = SIG / r02
        return r1 * r1 * r2 * r2 * math.exp(-ua2 - 0.5 * H * x2 * x2 - u * (s ** 12 - 2 * s ** 6))

    opts = dict(epsabs=1e-13, epsrel=1e-8)
    lim = (R0 - xmax, R0 + xmax, R0 - 1.0, R0 + 1.0, -1, 1)
    Z = integrate.tplquad(lambda c, r2, r1: weight(r1, r2, c), *lim, **opts)[0]
    want = {k: integrate.tplquad(lambda c, r2, r1: f(r1, r2, c) * weight(r1, r2, c), *lim, **opts)[0] / Z
            for k, f in (("cos", lambda r1, r2, c: c), ("r1", lambda r1, r2, c: r1),
                         ("r2", lambda r1, r2, c: r2))}
    C, R, dt, steps = 512, 8, 2e-3, 40000
    chains = [I.Chain(n_beads=3, n_replicas=R, spring=I.SPRING_VWF, H=H, r0=R0, lj_u=u, lj_sigma=SIG,
                      vwf_fa=fa, vwf_fb=fb, vwf_xmax=xmax, hi_a=1.0) for _ in range(C)]
    pos0 = np.zeros((3 * C, 3))
    pos0[:, 2] = np.tile([0.0, 2.0, 4.0], C)
    ctx = bdra.Context(chains, dt, steps, 35, pos0, precision=bdra.BD_PREC_FP32, max_windows=1,
                       stream=torch.cuda.current_stream().cuda_stream)
    ctx.step(steps)
    allpos = ctx.positions(True).reshape(C, R + 1, 3, 3)
    assert ctx.info().overextensions == 0
    ctx.close()
    q1, q2 = allpos[:, :, 1] - allpos[:, :, 0], allpos[:, :, 2] - allpos[:, :, 1]
    n1, n2 = np.linalg.norm(q1, axis=-1).ravel(), np.linalg.norm(q2, axis=-1).ravel()
    cos_bead = (-(q1 * q2).sum(axis=-1)).ravel() / (n1 * n2)
    for est, key in ((cos_bead, "cos"), (n1, "r1"), (n2, "r2")):
        sd = est.std() / math.sqrt(est.size)
        assert abs(est.mean() - want[key]) < 5 * sd + 0.003 * abs(want[key]), (key, est.mean(), want[key], sd)
