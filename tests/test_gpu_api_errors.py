"""Argument and state errors of the C ABI on a live context: each call fails
with its documented status before launching anything and leaves the context
as it was (a failed call keeps the previous state), and the context stays
usable afterwards.

- bd_step: 0 steps is a no-op; a negative count is BD_E_INVALID; a run past
  max_windows is BD_E_CAPACITY.
- bd_replica_average / bd_time_average: a window that has not completed (or
  a negative index) is BD_E_INVALID.
- bd_set_positions: a step that is not a window start is BD_E_INVALID; one
  past max_windows is BD_E_CAPACITY; a window start is accepted.
"""
import numpy as np
import pytest

from paper_2206_05851_gb300 import bdra
from paper_2206_05851_gb300 import inputs as I

pytestmark = pytest.mark.gpu

S, DT = 10, 1e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2206_05851_gb300 import build as B
    B.build()
    torch.cuda.init()


def _ctx():
    import torch
    ch = [I.Chain(n_beads=5, n_replicas=4, spring=I.SPRING_FENE, b=20.0, flow=I.FLOW_UNIAXIAL, rate=0.5)]
    pos0 = I.initial_positions(I.custom(ch, DT, S, 3 * S), seed=2)
    ctx = bdra.Context(ch, DT, S, 7, pos0, precision=bdra.BD_PREC_FP64, max_windows=3,
                       stream=torch.cuda.current_stream().cuda_stream)
    return ctx, pos0


def _raises(status, fn, *args):
    with pytest.raises(bdra.BdError) as e:
        fn(*args)
    assert e.value.status == status


def test_step_counts():
    ctx, _ = _ctx()
    ctx.step(12)
    before = ctx.positions(True)
    launches = ctx.info().kernel_launches
    ctx.step(0)
    _raises(bdra.BD_E_INVALID, ctx.step, -1)
    _raises(bdra.BD_E_CAPACITY, ctx.step, 30)          # to step 42: 4 windows, max_windows 3
    info = ctx.info()
    assert info.step == 12 and info.kernel_launches == launches
    np.testing.assert_array_equal(ctx.positions(True), before)
    ctx.step(18)                                        # to step 30: still usable
    assert ctx.info().windows_done == 3
    ctx.close()


def test_window_queries_and_restart_steps():
    ctx, pos0 = _ctx()
    ctx.step(2 * S)
    rsf, tsf = ctx.replica_average(1), ctx.time_average(1)
    assert np.isfinite(rsf).all() and np.isfinite(tsf).all()
    for w in (-1, 2):
        _raises(bdra.BD_E_INVALID, ctx.replica_average, w)
        _raises(bdra.BD_E_INVALID, ctx.time_average, w)
    before = ctx.positions(True)
    _raises(bdra.BD_E_INVALID, ctx.set_positions, pos0, S + 5)     # not a window start
    _raises(bdra.BD_E_CAPACITY, ctx.set_positions, pos0, 4 * S)    # past max_windows
    assert ctx.info().step == 2 * S
    np.testing.assert_array_equal(ctx.positions(True), before)
    np.testing.assert_array_equal(ctx.replica_average(1), rsf)
    ctx.set_positions(pos0, S)                                     # a window start
    assert ctx.info().step == S and ctx.info().windows_done == 1
    ctx.close()
