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


def _numpy_compaction(ft, fb, offs):
    """The event list written out plainly: springs in order, then criterion,
    then kind (threshold before Bell)."""
    M = ft.shape[1]
    steps = np.stack([ft.T, fb.T], axis=2)               # [M][3][2]
    m, q, kind = np.nonzero(steps >= 0)
    chain = np.searchsorted(offs, m, side="right") - 1
    out = np.zeros(len(m), dtype=bdra.EVENT_DTYPE)
    out["chain"], out["spring"], out["criterion"], out["kind"] = chain, m - offs[chain], q, kind
    out["step"] = steps[m, q, kind]
    assert M == offs[-1]
    return out


def test_noalloc_compaction_at_its_maximum_size_with_truncation():
    # 2^20 springs (the scratch's limit: 4096 blocks, so the single-block scan
    # carries over 16 passes) over many chains of uneven length, synthetic
    # first-event arrays; then a capacity below the total, where the count
    # must still be the full one and the first `capacity` events written
    import torch
    rng = np.random.default_rng(11)
    M = bdra.NOALLOC_MAX_SPRINGS
    lens = rng.integers(1, 600, size=4000)
    lens = lens[np.cumsum(lens) < M]
    lens = np.append(lens, M - lens.sum())
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    C = len(lens)
    ft = np.where(rng.random((3, M)) < 0.02, rng.integers(0, 10**6, size=(3, M)), -1).astype(np.int64)
    fb = np.where(rng.random((3, M)) < 0.01, rng.integers(0, 10**6, size=(3, M)), -1).astype(np.int64)
    want = _numpy_compaction(ft, fb, offs)
    stream = torch.cuda.current_stream().cuda_stream
    d_ft, d_fb = torch.from_numpy(ft).cuda(), torch.from_numpy(fb).cuda()
    d_offs = torch.from_numpy(offs).cuda()
    for cap in (len(want) + 5, len(want) // 3):
        out = torch.full((cap * 24,), 0xAB, dtype=torch.uint8, device="cuda")
        n_out = torch.full((1,), -7, dtype=torch.int64, device="cuda")
        bdra.bd_compact_events_noalloc(d_ft, d_fb, M, d_offs, C, out, cap, n_out, stream)
        torch.cuda.synchronize()
        assert int(n_out.item()) == len(want)
        got = np.frombuffer(out.cpu().numpy().tobytes(), dtype=bdra.EVENT_DTYPE)
        k = min(cap, len(want))
        np.testing.assert_array_equal(got[:k], want[:k])
        if cap > len(want):                  # nothing written past the events
            assert (out.cpu().numpy()[len(want) * 24:] == 0xAB).all()
