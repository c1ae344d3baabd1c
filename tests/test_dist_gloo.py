"""The multi-GPU host logic on two CPU ranks (gloo): each rank's own block of
cells, the max over ranks of the timed region, and the whole-job value."""
import os

import numpy as np
import torch.multiprocessing as mp

from paper_2511_21031_gb300 import dist as pdist
from paper_2511_21031_gb300 import workloads


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, lr = pdist.env_rank()
    wl = workloads.config_grid128(seed=pdist.rank_seed(2, r), edge=8)
    local_ms = 10.0 * (r + 1)                      # rank 1 is the slowest
    ms = pdist.max_over_ranks(local_ms)
    val = pdist.weak_scaling_value(wl.bins_total * 5, ms, ws)
    out[r] = (ws, r, lr, float(wl.theta[:4].sum()), ms, val, wl.bins_total)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_cells_and_take_the_slowest_time():
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    (ws0, r0, _, th0, ms0, v0, n0), (ws1, r1, _, th1, ms1, v1, n1) = res[0], res[1]
    assert ws0 == ws1 == 2 and (r0, r1) == (0, 1)
    assert th0 != th1                                # different cells (seeds) per rank
    assert n0 == n1                                  # same work per rank: weak scaling
    assert ms0 == ms1 == 20.0                        # max over ranks
    assert v0 == v1 == n0 * 5 * 2 / 20e-3


def test_single_process_helpers():
    assert pdist.env_rank() == (1, 0, 0) or "WORLD_SIZE" in os.environ
    assert pdist.max_over_ranks(3.5) == 3.5
    assert pdist.rank_seed(2, 0) == 2 and pdist.rank_seed(2, 3) == 3002
    assert np.isclose(pdist.weak_scaling_value(100, 10.0, 4), 40000.0)
