"""GPU parity for the paper's collapsed-chain model (Sec. II): harmonic springs
with rest length 2a and Lennard-Jones cohesion between non-adjacent beads, in
the paper's units mapped to the Hookean ones of the library (length a,
energy kT, bead diffusivity 1/4, so that tau is 4 time units and a shear rate
gamma-dot / tau is gamma-dot / 4).

- Same seeded inputs and Philox draws as the FP64 oracle: parent and replica
  positions, RSF and TSF profiles (per chain and window) within 1e-10 (FP64)
  / 1e-4 (FP32) relative; FP64 first-event steps (signed Eq. 4 force against
  the threshold, Bell hazards) equal; FP32 first-event steps equal except at
  near-ties checked against the oracle's own force or hazard at their step.
- Every collapsed-chain tile (2, 4, 5, 7, 16 springs per lane), ragged slots,
  the two-bead chain (no pair), a harmonic chain without cohesion, and a
  FENE chain in the same batch.
- Identical noise: the replicas follow the parent (their positions come from
  the same bonds by a differently blocked prefix sum, so to rounding only).
- The Eq. 5 diagnostics of collapsed chains against the oracle's.
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
DT, S, STEPS = 4e-5, 50, [30, 170, 200]       # tau_paper = 1e-5 per step; calls end mid-window


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2206_05851_gb300 import build as B
    B.build()
    torch.cuda.init()


def _collapsed(N, R, flow=I.FLOW_NONE, rate=0.0, u=1.0):
    return I.Chain(n_beads=N, n_replicas=R, spring=I.SPRING_HARMONIC, flow=flow, rate=rate,
                   H=400.0, r0=2.0, lj_u=u, lj_sigma=2.0, f_c=30.0, k0=50.0, dx=0.1)


def _chains():
    return [_collapsed(50, 16, I.FLOW_SHEAR, 7.5),           # the paper's chain at gamma-dot 30
            _collapsed(12, 5),
            _collapsed(48, 9, I.FLOW_PLANAR, 1.0),                # five springs per lane
            _collapsed(3, 3, I.FLOW_UNIAXIAL, 2.0),
            _collapsed(120, 6, I.FLOW_PLANAR, 1.0),
            _collapsed(300, 3, I.FLOW_SHEAR, 7.5),
            _collapsed(2, 2, I.FLOW_SHEAR, 7.5),
            _collapsed(7, 4, I.FLOW_SHEAR, 7.5, u=0.0),
            I.Chain(n_beads=20, n_replicas=8, spring=I.SPRING_FENE, flow=I.FLOW_UNIAXIAL, b=50.0,
                    rate=0.5, f_c=5.0, k0=1e-2, dx=0.2)]


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def _gpu(chains, pos0, prec, seed=7, flags=0, thr=7, bell=7):
    total = sum(STEPS)
    ctx = bdra.Context(chains, DT, S, seed, pos0, precision=prec, max_windows=total // S + 1,
                       thr_mask=thr, bell_mask=bell, flags=flags, stream=_stream())
    for n in STEPS:
        ctx.step(n)
    nw = total // S
    out = dict(pos=ctx.positions(False), allpos=ctx.positions(True),
               rsf=np.array([ctx.replica_average(w) for w in range(nw)]).reshape(nw, ctx.M),
               tsf=np.array([ctx.time_average(w) for w in range(nw)]).reshape(nw, ctx.M))
    out["haz"], out["first_thr"], out["first_bell"] = ctx.kinetics()
    if flags & bdra.BD_FLAG_CONFORMATION:
        conf = [ctx.conformation(w) for w in range(nw)]
        out["conf"] = tuple(np.array([c[k] for c in conf]) for k in range(3))
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


@pytest.fixture(scope="module")
def oracle_run():
    chains = _chains()
    pos0 = I.initial_positions(I.custom(chains, DT, S, sum(STEPS)), seed=23)
    r = O.run(chains, DT, S, sum(STEPS), 7, pos0, thr_mask=7, bell_mask=7, n_threads=8)
    return chains, pos0, r


def test_initial_conformations_have_no_overlap(oracle_run):
    chains, pos0, _ = oracle_run
    o = 0
    for c in chains:
        r = pos0[o:o + c.n_beads]
        o += c.n_beads
        if c.lj_u > 0 and c.n_beads > 2:
            d = np.linalg.norm(r[:, None] - r[None], axis=2)
            iu = np.triu_indices(c.n_beads, 2)
            assert d[iu].min() > 0.9 * c.lj_sigma


@pytest.mark.parametrize("prec", PRECS)
def test_collapsed_chains_match_oracle(oracle_run, prec):
    chains, pos0, r = oracle_run
    g = _gpu(chains, pos0, prec)
    tol = TOL[prec]
    nb = [c.n_beads for c in chains]
    assert _rel(g["pos"], O.com_frame(r["pos"], nb), nb) <= tol
    par, rep = _split(g["allpos"], chains)
    np.testing.assert_array_equal(par, g["pos"])
    sizes = [c.n_beads for c in chains for _ in range(c.n_replicas)]
    assert _rel(rep, O.com_frame(r["rep"], sizes), sizes) <= tol
    PE.check_profiles(g, r, chains, tol)
    # the profiles are signed: compressed springs (f < 0) are sampled too
    assert (r["rsf"] < 0).any() and (r["rsf"] > 0).any()
    assert (r["first_thr"] >= 0).sum() > 5 and (r["first_bell"] >= 0).sum() > 5
    if prec == bdra.BD_PREC_FP64:
        np.testing.assert_array_equal(g["first_thr"], r["first_thr"])
        np.testing.assert_array_equal(g["first_bell"], r["first_bell"])
        np.testing.assert_allclose(g["haz"], r["lam"], rtol=1e-9, atol=1e-300)
    else:
        replay = PE.OracleReplay(chains, DT, S, 7, pos0, 7, 7)
        PE.compare_events_fp32(g, r, chains, S, replay)
        PE.compare_hazards_fp32(g["haz"], r["lam"])


@pytest.mark.parametrize("prec", PRECS)
def test_identical_noise_replicas_follow_parent(prec):
    chains = _chains()
    pos0 = I.initial_positions(I.custom(chains, DT, S, sum(STEPS)), seed=4)
    g = _gpu(chains, pos0, prec, flags=bdra.BD_FLAG_IDENTICAL_NOISE, thr=0, bell=0)
    par, rep = _split(g["allpos"], chains)
    tol = 1e-11 if prec == bdra.BD_PREC_FP64 else 1e-4
    o = po = 0
    for ch in chains:
        p = par[po:po + ch.n_beads]
        for k in range(ch.n_replicas):
            x = rep[o + k * ch.n_beads:o + (k + 1) * ch.n_beads]
            assert np.abs(x - p).max() <= tol * np.abs(p).max()
        o += ch.n_replicas * ch.n_beads
        po += ch.n_beads


@pytest.mark.parametrize("prec", PRECS)
def test_collapsed_conformation_diagnostics(oracle_run, prec):
    chains, pos0, _ = oracle_run
    g = _gpu(chains, pos0, prec, flags=bdra.BD_FLAG_CONFORMATION, thr=0, bell=0)
    want = O.conformation(chains, DT, S, sum(STEPS), 7, pos0)
    for got, w in zip(g["conf"], want):
        assert np.abs(got - w).max() <= TOL[prec] * np.abs(w).max()


@pytest.mark.parametrize("prec", PRECS)
def test_longest_collapsed_chain(prec):
    # the maximum bead count (512: 16 springs per lane, 32 lanes per slot)
    ch = [_collapsed(512, 3, I.FLOW_SHEAR, 7.5)]
    pos0 = I.initial_positions(I.custom(ch, DT, 10, 30), seed=8)
    r = O.run(ch, DT, 10, 30, 3, pos0, thr_mask=7, bell_mask=7, n_threads=4)
    import torch
    ctx = bdra.Context(ch, DT, 10, 3, pos0, precision=prec, max_windows=4, thr_mask=7, bell_mask=7,
                       stream=torch.cuda.current_stream().cuda_stream)
    ctx.step(30)
    pos = ctx.positions(False)
    g = {"rsf": np.array([ctx.replica_average(w) for w in range(3)]),
         "tsf": np.array([ctx.time_average(w) for w in range(3)])}
    ctx.close()
    assert _rel(pos, O.com_frame(r["pos"], [512]), [512]) <= TOL[prec]
    PE.check_profiles(g, r, ch, TOL[prec])


def test_full_size_workloads_on_sampled_chains():
    # the bench's launch configurations (1024 collapsed chains; 128 with
    # hydrodynamic interaction; 64 vWF chains), float32, 300 steps; sampled
    # chains re-run alone by the oracle with their own chain ids in the noise
    # counter: positions per chain, RSF and TSF per (chain, window) row
    import torch
    for wl, sample in ((I.collapsed_1024(n_steps=300), [0, 611, 1023]),
                       (I.collapsed_hi_128(n_steps=300), [5, 127]),
                       (I.vwf_64(n_steps=300), [0, 63])):
        S = 100
        pos0 = I.initial_positions(wl)
        ctx = bdra.Context(wl.chains, wl.dt, S, wl.seed, pos0, precision=bdra.BD_PREC_FP32,
                           max_windows=4, thr_mask=wl.thr_mask, bell_mask=wl.bell_mask,
                           stream=torch.cuda.current_stream().cuda_stream)
        ctx.step(300)
        pos = ctx.positions(False)
        rsf = np.array([ctx.replica_average(w) for w in range(3)])
        tsf = np.array([ctx.time_average(w) for w in range(3)])
        ctx.close()
        boff = I.bead_offsets(wl.chains)
        soff = I.spring_offsets(wl.chains)
        sub = [wl.chains[c] for c in sample]
        sub_pos = np.concatenate([pos0[boff[c]:boff[c + 1]] for c in sample])
        r = O.run(sub, wl.dt, S, 300, wl.seed, sub_pos, thr_mask=wl.thr_mask, bell_mask=wl.bell_mask,
                  n_threads=8, chain_ids=sample)
        got = np.concatenate([pos[boff[c]:boff[c + 1]] for c in sample])
        nb = [c.n_beads for c in sub]
        assert _rel(got, O.com_frame(r["pos"], nb), nb) <= 1e-4, wl.name
        g = {k: np.concatenate([v[:, soff[c]:soff[c + 1]] for c in sample], axis=1)
             for k, v in (("rsf", rsf), ("tsf", tsf))}
        PE.check_profiles(g, r, sub, 1e-4)
