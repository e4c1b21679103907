"""Failure detection of the tensor-core kernels, without a GPU fault.

The float32 kernels with hydrodynamic interaction (chains of up to 50 beads)
wait on completion barriers of their own MMAs, every wait bounded. With
BD_FLAG_TEST_TC_STALL they issue no MMA and no completion, so the waits give
up (about a second each): each CTA records the failure in the context's device
error word, stops integrating and frees its tensor memory. The calls that read
the word (bd_get_info, bd_detect_events) then return BD_E_TIMEOUT, and the GPU
stays usable: a context created afterwards runs and matches the oracle.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2206_05851_gb300 import bdra
from paper_2206_05851_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DT, S, STEPS = 4e-5, 5, 10


def _chains():
    # the paper's collapsed chain with RPY, 12 beads: two 32-column panels
    return [I.Chain(n_beads=12, n_replicas=2, spring=I.SPRING_HARMONIC, flow=I.FLOW_SHEAR, rate=7.5,
                    H=400.0, r0=2.0, lj_u=1.0, lj_sigma=2.0, f_c=30.0, k0=50.0, dx=0.1, hi_a=1.0)]


def _ctx(chains, pos0, flags):
    import torch
    return bdra.Context(chains, DT, S, 9, pos0, precision=bdra.BD_PREC_FP32,
                        max_windows=STEPS // S + 1, flags=flags,
                        stream=torch.cuda.current_stream().cuda_stream)


def test_stalled_waits_report_timeout_and_the_gpu_stays_usable():
    chains = _chains()
    pos0 = I.initial_positions(I.custom(chains, DT, S, STEPS), seed=3)
    ctx = _ctx(chains, pos0, bdra.BD_FLAG_TEST_TC_STALL)
    ctx.step(STEPS)
    with pytest.raises(bdra.BdError) as e:
        ctx.info()
    assert e.value.status == bdra.BD_E_TIMEOUT
    with pytest.raises(bdra.BdError) as e:
        ctx.events()
    assert e.value.status == bdra.BD_E_TIMEOUT
    ctx.close()

    ctx = _ctx(chains, pos0, 0)
    ctx.step(STEPS)
    info = ctx.info()
    assert info.step == STEPS
    got = ctx.positions()
    ctx.close()
    ref = O.run(chains, DT, S, STEPS, 9, pos0, thr_mask=0, bell_mask=0)
    want = O.com_frame(ref["pos"], [c.n_beads for c in chains])
    assert np.abs(got - want).max() / np.abs(want).max() <= 1e-4
