"""One workload split into contiguous chain ranges over several contexts,
each with its range's first global chain index as chain_id_base (the
multi-GPU form of the method, here as consecutive contexts on one GPU: the
contexts never wait on each other). The union of their results must equal
the whole workload in one context bit for bit: parent and replica
positions, RSF and TSF histories, Bell hazards, first events, the event
list (with global chain indices) and the log-survival; and, for FENE chains
with checkpoints, the adjoint's gradients. Free-draining FENE and Hookean
chains, a collapsed chain (Lennard-Jones kernels) and a chain with RPY
hydrodynamic interaction, in both precisions; and the oracle run of a
range with its global chain ids."""
import numpy as np
import pytest

import parity_events as PE
from oracle import oracle as O
from paper_2206_05851_gb300 import bdra, shard
from paper_2206_05851_gb300 import inputs as I

pytestmark = pytest.mark.gpu

PRECS = [bdra.BD_PREC_FP64, bdra.BD_PREC_FP32]
DT, S, N_STEPS, SEED = 1e-3, 10, 60, 21


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2206_05851_gb300 import build as B
    B.build()
    torch.cuda.init()


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def _chains(with_models: bool):
    out = []
    for k, (n, R) in enumerate([(30, 8), (6, 3), (100, 16), (40, 2), (9, 5), (20, 40), (3, 7)]):
        b = 30.0 + 5 * k
        out.append(I.Chain(n_beads=n, n_replicas=R, spring=I.SPRING_FENE if k % 3 else I.SPRING_HOOKE,
                           flow=(I.FLOW_UNIAXIAL, I.FLOW_SHEAR, I.FLOW_PLANAR)[k % 3], b=b,
                           rate=0.3 + 0.1 * k, f_c=0.3 * b ** 0.5, k0=0.5, dx=0.5))
    if with_models:
        col = I.collapsed_chain(3, n_beads=12)
        col.f_c, col.k0, col.dx = 30.0, 5.0, 0.1
        hi = I.collapsed_chain(2, n_beads=10)
        hi.hi_a, hi.f_c, hi.k0, hi.dx = 1.0, 30.0, 5.0, 0.1
        out[2:2] = [col]
        out.append(hi)
    return out


def _run(chains, pos0, prec, base, dt=DT, checkpoint=0):
    ctx = bdra.Context(chains, dt, S, SEED, pos0, precision=prec, max_windows=N_STEPS // S,
                       thr_mask=7, bell_mask=7, stream=_stream(), chain_id_base=base,
                       checkpoint_steps=checkpoint)
    ctx.step(N_STEPS)
    nw = N_STEPS // S
    out = dict(pos=ctx.positions(False), allpos=ctx.positions(True),
               rsf=np.array([ctx.replica_average(w) for w in range(nw)]).reshape(nw, ctx.M),
               tsf=np.array([ctx.time_average(w) for w in range(nw)]).reshape(nw, ctx.M))
    out["haz"], out["first_thr"], out["first_bell"] = ctx.kinetics()
    ev, ls = ctx.events()
    out["events"], out["log_surv"] = shard.globalize_events(ev, base), ls
    if checkpoint:
        rng = np.random.default_rng(3)
        G = rng.normal(size=(nw, ctx.M))
        out["G"] = G
    return ctx, out


def _join(parts, key, axis):
    return np.concatenate([p[key] for p in parts], axis=axis)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("world", [2, 3])
def test_split_contexts_equal_the_whole_workload(prec, world):
    chains = _chains(with_models=True)
    dt = I.COLLAPSED_DT
    pos0 = I.initial_positions(I.custom(chains, dt, S, N_STEPS), seed=4)
    ctx, whole = _run(chains, pos0, prec, 0, dt=dt)
    ctx.close()
    parts = []
    for r in range(world):
        sub, p0, base = shard.rank_share(chains, pos0, r, world)
        c, out = _run(sub, p0, prec, base, dt=dt)
        c.close()
        parts.append(out)
    for key, axis in (("pos", 0), ("allpos", 0), ("rsf", 1), ("tsf", 1), ("haz", 1),
                      ("first_thr", 1), ("first_bell", 1), ("events", 0), ("log_surv", 0)):
        np.testing.assert_array_equal(_join(parts, key, axis), whole[key], err_msg=key)
    assert len(whole["events"]) > 10


def test_split_contexts_give_the_whole_workloads_gradients():
    chains = _chains(with_models=False)
    pos0 = I.initial_positions(I.custom(chains, DT, S, N_STEPS), seed=6)
    ctx, whole = _run(chains, pos0, bdra.BD_PREC_FP64, 0, checkpoint=2 * S)
    gls = np.linspace(-1.0, 1.0, len(chains))
    g_whole = ctx.adjoint(whole["G"], gls)
    ctx.close()
    offs = I.spring_offsets(chains)
    got = []
    for r in range(2):
        sub, p0, base = shard.rank_share(chains, pos0, r, 2)
        c, _ = _run(sub, p0, bdra.BD_PREC_FP64, base, checkpoint=2 * S)
        cols = slice(offs[base], offs[base + len(sub)])
        got.append(c.adjoint(np.ascontiguousarray(whole["G"][:, cols]), gls[base:base + len(sub)]))
        c.close()
    # float64 gradient partials meet in atomics: equal up to their order
    np.testing.assert_allclose(np.concatenate(got), g_whole, rtol=1e-12, atol=1e-300)


def test_range_matches_the_oracle_with_global_chain_ids():
    chains = _chains(with_models=False)
    pos0 = I.initial_positions(I.custom(chains, DT, S, N_STEPS), seed=8)
    sub, p0, base = shard.rank_share(chains, pos0, 1, 2)
    assert base > 0
    ctx, g = _run(sub, p0, bdra.BD_PREC_FP64, base)
    ctx.close()
    r = O.run(sub, DT, S, N_STEPS, SEED, p0, thr_mask=7, bell_mask=7,
              chain_ids=list(range(base, base + len(sub))))
    nb = [c.n_beads for c in sub]
    want = O.com_frame(r["pos"], nb)
    assert np.abs(g["pos"] - want).max() / np.abs(want).max() <= 1e-10
    PE.check_profiles(g, r, sub, 1e-10)
    np.testing.assert_array_equal(g["first_thr"], r["first_thr"])
    np.testing.assert_array_equal(g["first_bell"], r["first_bell"])
    # and the same range without the base draws other noise
    ctx, g0 = _run(sub, p0, bdra.BD_PREC_FP64, 0)
    ctx.close()
    assert not np.allclose(g0["rsf"], g["rsf"])
