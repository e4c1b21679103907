"""The allocation-free event compaction, bd_compact_events_noalloc, against
the event list of bd_detect_events, through the C ABI.

The allocation-free call exists for callers that may not allocate device
memory when they need the events: code running while a stream is captured
into a CUDA graph, an engine that owns a fixed device-memory arena, or a
real-time loop that must not wait on the allocator. Its scratch is a fixed
device array inside the library, so the test also checks that a second call
(which overwrites the first call's scratch) is still exact.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes when run alone.
"""
import math

import numpy as np
import pytest

from paper_2206_05851_gb300 import bdra
from paper_2206_05851_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _chains():
    b = 30.0
    return [I.Chain(n_beads=16, n_replicas=24, spring=I.SPRING_FENE, flow=I.FLOW_UNIAXIAL,
                    b=b, rate=0.8, f_c=0.55 * math.sqrt(b), k0=1e-4, dx=8.0 / math.sqrt(b)),
            I.Chain(n_beads=40, n_replicas=12, spring=I.SPRING_FENE, flow=I.FLOW_SHEAR,
                    b=b, rate=3.0, f_c=0.5 * math.sqrt(b), k0=1e-4, dx=8.0 / math.sqrt(b)),
            I.Chain(n_beads=300, n_replicas=5, spring=I.SPRING_FENE, flow=I.FLOW_PLANAR,
                    b=b, rate=0.2, f_c=0.45 * math.sqrt(b), k0=1e-4, dx=4.0 / math.sqrt(b))]


def test_noalloc_compaction_matches_detect_events_on_consecutive_calls():
    import torch
    from paper_2206_05851_gb300 import build as B
    B.build()
    torch.cuda.init()
    stream = torch.cuda.current_stream().cuda_stream
    chains = _chains()
    S, dt = 20, 2e-3
    pos0 = I.initial_positions(I.custom(chains, dt, S, 2000), seed=8)
    ctx = bdra.Context(chains, dt, S, 3, pos0, precision=bdra.BD_PREC_FP32, max_windows=100,
                       thr_mask=7, bell_mask=7, stream=stream)
    M, C = ctx.M, len(chains)
    spr_off = torch.from_numpy(I.spring_offsets(chains)).cuda()
    cap = 6 * M
    counts = []
    for n_steps in (600, 1400):
        ctx.step(n_steps)
        ref, _ = ctx.events(capacity=cap)              # bd_detect_events
        haz = torch.zeros((3, M), dtype=torch.float64, device="cuda")
        ft = torch.zeros((3, M), dtype=torch.int64, device="cuda")
        fb = torch.zeros((3, M), dtype=torch.int64, device="cuda")
        bdra.bd_get_kinetics(ctx.ptr, haz, ft, fb)
        out = torch.full((cap * 24,), 0xAB, dtype=torch.uint8, device="cuda")
        n_out = torch.full((1,), -7, dtype=torch.int64, device="cuda")
        bdra.bd_compact_events_noalloc(ft, fb, M, spr_off, C, out, cap, n_out, stream)
        torch.cuda.synchronize()
        n = int(n_out.item())
        got = np.frombuffer(out.cpu().numpy().tobytes(), dtype=bdra.EVENT_DTYPE)[:n]
        assert n == len(ref)
        np.testing.assert_array_equal(got, ref)
        counts.append(n)
    assert 0 < counts[0] < counts[1]
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    dummy = torch.zeros(8, dtype=torch.int64, device="cuda")
    with pytest.raises(bdra.BdError) as e:
        bdra.bd_compact_events_noalloc(dummy, dummy, bdra.NOALLOC_MAX_SPRINGS + 1, dummy, 1,
                                       dummy, 0, dummy)
    assert e.value.status == bdra.BD_E_CAPACITY
