"""Conformation diagnostics of Eq. 5 on the GPU (bd_conformation) against the
oracle's on the same seeded inputs and Philox draws: the per-replica
bead-mean difference between each replica after the evolution time and the
halted parent, its replica-averaged per-bead form, and the parent's R_GZ.
FP64 within 1e-10 relative to the largest value of each output; FP32 within
1e-4 (the float32 trajectories' deviation, measured at the FP64 oracle's
scale). Both replica layouts, several tiles, windows that span step calls."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2206_05851_gb300 import bdra
from paper_2206_05851_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2206_05851_gb300 import build as B
    B.build()
    torch.cuda.init()


def _chains():
    return [I.Chain(n_beads=6, n_replicas=40, spring=I.SPRING_FENE, flow=I.FLOW_SHEAR, b=30.0, rate=1.0),
            I.Chain(n_beads=100, n_replicas=9, spring=I.SPRING_FENE, flow=I.FLOW_PLANAR, b=100.0, rate=0.05),
            I.Chain(n_beads=2, n_replicas=3, spring=I.SPRING_HOOKE, flow=I.FLOW_UNIAXIAL, rate=0.2),
            I.Chain(n_beads=37, n_replicas=17, spring=I.SPRING_FENE, flow=I.FLOW_UNIAXIAL, b=50.0, rate=0.1)]


def _gpu(chains, dt, S, steps, seed, pos0, prec, layout=0, lanes=0):
    import torch
    ctx = bdra.Context(chains, dt, S, seed, pos0, precision=prec,
                       max_windows=sum(steps) // S + 1, flags=bdra.BD_FLAG_CONFORMATION,
                       stream=torch.cuda.current_stream().cuda_stream, layout_hint=layout,
                       lanes_hint=lanes)
    for n in steps:
        ctx.step(n)
    W = sum(steps) // S
    out = [ctx.conformation(w) for w in range(W)]
    ctx.close()
    return (np.array([o[0] for o in out]), np.array([o[1] for o in out]),
            np.array([o[2] for o in out]))


def _close(got, want, rtol):
    for g, w in zip(got, want):
        scale = np.abs(w).max()
        err = np.abs(g - w).max()
        assert err <= rtol * scale, (err, scale)


@pytest.mark.parametrize("prec,layout", [(bdra.BD_PREC_FP64, 0), (bdra.BD_PREC_FP32, 1),
                                         (bdra.BD_PREC_FP32, 2)])
def test_conformation_matches_oracle(prec, layout):
    chains = _chains()
    dt, S = 2e-3, 25
    pos0 = I.initial_positions(I.custom(chains, dt, S, 100), seed=51)
    want = O.conformation(chains, dt, S, 100, 7, pos0, n_threads=4)
    got = _gpu(chains, dt, S, [30, 45, 25], 7, pos0, prec, layout=layout)   # windows span the calls
    _close(got, want, 1e-10 if prec == bdra.BD_PREC_FP64 else 1e-4)
    assert np.all(want[0] > 0) and np.all(want[2] > 0)


def test_conformation_needs_the_flag():
    import torch
    chains = _chains()[:1]
    pos0 = I.initial_positions(I.custom(chains, 1e-3, 10, 10), seed=1)
    ctx = bdra.Context(chains, 1e-3, 10, 0, pos0, max_windows=2,
                       stream=torch.cuda.current_stream().cuda_stream)
    ctx.step(10)
    with pytest.raises(bdra.BdError) as e:
        ctx.conformation(0)
    assert e.value.status == bdra.BD_E_STATE
    ctx.close()
