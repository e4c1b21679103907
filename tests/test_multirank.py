"""The multi-GPU (weak-scaling) host logic on CPU: two gloo ranks, each with
its own chain set of the workload's shape, no collective on the data path,
the timed interval taken as the maximum over ranks.

Each rank integrates its chains with the FP64 oracle (standing in for its
GPU: the host logic is the same), so the test also shows that a rank's
results depend only on its own keys - running it alone gives the same
numbers - and that the ranks draw different noise."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2206_05851_gb300 import inputs as I
from paper_2206_05851_gb300 import shard

WORLD = 2
STEPS, CHAINS = 60, 2


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_run(wl, rank):
    from oracle import oracle as O
    seed, init_seed = shard.rank_keys(wl.seed, wl.init_seed, rank)
    pos0 = I.initial_positions(wl, seed=init_seed)
    r = O.run(wl.chains, wl.dt, wl.window_steps, STEPS, seed, pos0, thr_mask=0, bell_mask=0,
              want_replicas=False)
    return seed, r["rsf"]


def _worker(rank, port, out_dir):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    wl = I.planar_1024(n_steps=STEPS, n_chains=CHAINS)
    wl.window_steps = 20
    dist.barrier()
    seed, rsf = _rank_run(wl, rank)
    dist.barrier()
    t_local = 1.5 * (rank + 1)
    t_max = shard.max_over_ranks(t_local, dist)
    units = float(wl.bead_steps())
    rate = shard.whole_job_rate(units, WORLD, t_max)
    seeds = [None] * WORLD
    dist.all_gather_object(seeds, seed)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), rsf=rsf, t_max=t_max, rate=rate,
             units=units, seeds=np.array(seeds))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_chains_without_data_collectives(tmp_path):
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
    res = [np.load(tmp_path / f"rank{r}.npz") for r in range(WORLD)]
    # the slowest rank's time, seen by every rank; whole-job rate over it
    for r in res:
        assert float(r["t_max"]) == 1.5 * WORLD
        assert float(r["rate"]) == pytest.approx(float(r["units"]) * WORLD / (1.5 * WORLD))
    # distinct keys, distinct noise, identical to running each rank alone
    assert len(set(res[0]["seeds"].tolist())) == WORLD
    assert not np.allclose(res[0]["rsf"], res[1]["rsf"])
    wl = I.planar_1024(n_steps=STEPS, n_chains=CHAINS)
    wl.window_steps = 20
    for r in range(WORLD):
        _, alone = _rank_run(wl, r)
        np.testing.assert_array_equal(res[r]["rsf"], alone)


def test_rank_keys_and_rate_arguments():
    assert shard.rank_keys(5, 7, 0) == (5, 7)
    assert shard.rank_keys(5, 7, 3) == (5 + 3 * shard.RANK_SEED_STRIDE, 10)
    with pytest.raises(ValueError):
        shard.rank_keys(5, 7, -1)
    with pytest.raises(ValueError):
        shard.whole_job_rate(1.0, 2, 0.0)
    assert shard.max_over_ranks(2.5) == 2.5
