"""The multi-GPU host logic on CPU: one workload split over two gloo ranks.

Each rank integrates its contiguous range of the workload's chains (balanced
by N (R + 1)) with the global chain ids in the noise counter. The FP64 oracle
stands in for the rank's GPU (the host logic is the same; the GPU side of
the chain ids is tested in test_gpu_multicontext.py). After the integration,
and only then, the ranks gather their event lists, force-profile rows and
log-survival and sum a rupture-location histogram. Rank 0's gathered results
must equal, bit for bit, the whole workload run in one piece; the timed
interval is the maximum over ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2206_05851_gb300 import bdra
from paper_2206_05851_gb300 import inputs as I
from paper_2206_05851_gb300 import shard

WORLD = 2
STEPS, S = 60, 20


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _workload():
    # uneven chains with both criteria on, so that the split is not by count
    chains = []
    for k, (n, R) in enumerate([(30, 8), (6, 3), (12, 16), (40, 2), (9, 5), (20, 4), (3, 7)]):
        b = 30.0
        chains.append(I.Chain(n_beads=n, n_replicas=R, spring=I.SPRING_FENE, flow=I.FLOW_UNIAXIAL,
                              b=b, rate=0.6 + 0.1 * k, f_c=0.3 * b ** 0.5, k0=0.5, dx=0.5))
    wl = I.custom(chains, 2e-3, S, STEPS)
    wl.thr_mask = wl.bell_mask = 7
    return wl


def _events(first_thr, first_bell, chains):
    """Event list of first-event arrays [3][M], in (chain, spring, criterion,
    kind) order (the library's bd_detect_events order)."""
    offs = I.spring_offsets(chains)
    rows = []
    for c in range(len(chains)):
        for i in range(offs[c + 1] - offs[c]):
            for q in range(3):
                for kind, arr in ((0, first_thr), (1, first_bell)):
                    if arr[q, offs[c] + i] >= 0:
                        rows.append((c, i, q, kind, arr[q, offs[c] + i]))
    return np.array(rows, dtype=bdra.EVENT_DTYPE)


def _run(chains, pos0, chain_ids):
    from oracle import oracle as O
    wl = _workload()
    r = O.run(chains, wl.dt, S, STEPS, wl.seed, pos0, thr_mask=7, bell_mask=7,
              want_replicas=False, chain_ids=chain_ids)
    offs = I.spring_offsets(chains)
    log_surv = np.array([-r["lam"][:, offs[c]:offs[c + 1]].sum(axis=1) for c in range(len(chains))])
    # rupture location: the spring of each chain's first RSF threshold event
    hist = np.zeros(64)
    for c in range(len(chains)):
        t = r["first_thr"][2, offs[c]:offs[c + 1]]
        if (t >= 0).any():
            hist[int(np.argmin(np.where(t >= 0, t, np.iinfo(np.int64).max)))] += 1
    return r, _events(r["first_thr"], r["first_bell"], chains), log_surv, hist


def _worker(rank, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    wl = _workload()
    pos0 = I.initial_positions(wl)
    chains, p0, base = shard.rank_share(wl.chains, pos0, rank, WORLD)
    dist.barrier()
    r, ev, log_surv, hist = _run(chains, p0, list(range(base, base + len(chains))))
    dist.barrier()
    t_max = shard.max_over_ranks(1.5 * (rank + 1), dist)
    units = sum(ch.n_beads * ch.n_replicas for ch in chains) * STEPS
    units_all = shard.sum_counts(np.array([units]), dist)[0]
    events = shard.gather_events(shard.globalize_events(ev, base), dist)
    rsf = shard.gather_rows(r["rsf"], dist)
    tsf = shard.gather_rows(r["tsf"], dist)
    ls = shard.gather_rows(log_surv.T, dist)
    hist_all = shard.sum_counts(hist, dist)
    if rank == 0:
        np.savez(os.path.join(out_dir, "gathered.npz"), events=events, rsf=rsf, tsf=tsf, ls=ls,
                 hist=hist_all, t_max=t_max, rate=shard.whole_job_rate(units_all, t_max),
                 units_all=units_all)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), n_chains=len(chains), base=base, t_max=t_max)
    dist.destroy_process_group()


def test_two_gloo_ranks_split_one_workload_and_gather_the_whole_result(tmp_path):
    from oracle import oracle as O
    O.build()
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, str(tmp_path))) for r in range(WORLD)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    g = np.load(tmp_path / "gathered.npz")
    ranks = [np.load(tmp_path / f"rank{r}.npz") for r in range(WORLD)]
    wl = _workload()
    # contiguous, covering ranges; the slowest rank's time seen by every rank
    assert int(ranks[0]["base"]) == 0
    assert int(ranks[1]["base"]) == int(ranks[0]["n_chains"])
    assert sum(int(r["n_chains"]) for r in ranks) == len(wl.chains)
    for r in ranks:
        assert float(r["t_max"]) == 1.5 * WORLD
    assert float(g["units_all"]) == wl.bead_steps(STEPS)
    assert float(g["rate"]) == pytest.approx(wl.bead_steps(STEPS) / (1.5 * WORLD))
    # the union of the ranks is the whole workload in one piece, bit for bit
    whole, ev, log_surv, hist = _run(wl.chains, I.initial_positions(wl), None)
    assert len(ev) > 10
    np.testing.assert_array_equal(g["events"], ev)
    np.testing.assert_array_equal(g["rsf"], whole["rsf"])
    np.testing.assert_array_equal(g["tsf"], whole["tsf"])
    np.testing.assert_array_equal(g["ls"], log_surv.T)
    np.testing.assert_array_equal(g["hist"], hist)


def test_partition_is_contiguous_balanced_and_covering():
    costs = [5, 1, 1, 1, 9, 2, 2, 3, 8, 1]
    for world in range(1, len(costs) + 1):
        parts = shard.partition(costs, world)
        assert parts[0][0] == 0 and parts[-1][1] == len(costs)
        assert all(a < b for a, b in parts)
        assert all(parts[k][1] == parts[k + 1][0] for k in range(world - 1))
    # equal costs split evenly; one heavy chain gets a rank of its own
    assert shard.partition([1] * 8, 4) == [(0, 2), (2, 4), (4, 6), (6, 8)]
    assert shard.partition([1, 1, 100, 1, 1], 3)[1] == (2, 3)
    # balanced to within one chain of the ideal
    wl = I.uneven_4096(n_chains=512)
    cost = [shard.chain_cost(ch) for ch in wl.chains]
    for world in (2, 4, 8):
        loads = [sum(cost[a:b]) for a, b in shard.partition(cost, world)]
        assert max(loads) - sum(cost) / world <= max(cost)
    with pytest.raises(ValueError):
        shard.partition([1, 2], 3)
    with pytest.raises(ValueError):
        shard.rank_range(wl.chains, 2, 2)
    with pytest.raises(ValueError):
        shard.whole_job_rate(1.0, 0.0)
    assert shard.max_over_ranks(2.5) == 2.5
