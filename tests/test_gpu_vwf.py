"""GPU parity for the coarse-grained vWF chain (supplementary material, Table
S1, in the library's units): A2 domains (FENE in parallel with harmonic) on
the even springs, disulfide bonds on the odd springs, Lennard-Jones
cohesion, with and without RPY hydrodynamic interaction, against the FP64
oracle on the same seeded inputs and Philox draws.

- Positions of parents and replicas, RSF and TSF within 1e-10 (FP64) /
  1e-4 (FP32) relative; FP64 first-event steps and hazards equal (a raised
  unfolding rate, so that A2 domains unfold within the run).
- Disulfide bonds never have events and keep a zero hazard.
- Chains of 50 beads (the paper's), an odd bead count (a last A2 domain
  without a following bond), 7 beads with hydrodynamic interaction, and the
  two-bead chain (one A2 domain).
"""
import numpy as np
import pytest

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
    for got, want in ((rsf, r["rsf"]), (tsf, r["tsf"])):
        assert np.abs(got - want).max() / np.abs(want).max() <= tol
    offs = I.spring_offsets(chains)
    odd = np.concatenate([np.arange(offs[c] + 1, offs[c + 1], 2) for c in range(len(chains))])
    assert (first_thr[:, odd] < 0).all() and (first_bell[:, odd] < 0).all() and (haz[:, odd] == 0).all()
    if prec == bdra.BD_PREC_FP64:
        assert (r["first_bell"] >= 0).sum() > 10 and (r["first_thr"] >= 0).sum() > 10
        np.testing.assert_array_equal(first_thr, r["first_thr"])
        np.testing.assert_array_equal(first_bell, r["first_bell"])
        np.testing.assert_allclose(haz, r["lam"], rtol=1e-9, atol=1e-300)
    else:
        # float32: hazards in log space (a relative force error e moves k0 exp(dx f) by about dx f e)
        pos = r["lam"] > 0
        assert (np.abs(np.log(haz[pos]) - np.log(r["lam"][pos])) <= 1e-4 * np.abs(np.log(r["lam"][pos])) + 2e-3).all()
        np.testing.assert_array_equal(haz[~pos], r["lam"][~pos])
