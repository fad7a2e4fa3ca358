"""The N > 1 path of bench.py on CPU (gloo, world_size 2): each rank takes
a disjoint Philox shot range; only the timing (max) and the counts (sum)
are reduced.  Decoding each rank's shard (here with the oracle) gives the
same per-shot results as decoding all shots in one process."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

B_PER_RANK = 24


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    from oracle import codes

    H, _ = codes.build_code("planar", 5)
    shot0 = bench.shot_offset(rank, B_PER_RANK)
    ch = oracle.depolarizing(0.06)
    _, syn = oracle.sample(H, *ch, seed=bench.SEED, shot0=shot0, B=B_PER_RANK)
    est, conv, iters = oracle.decode(H, syn, np.tile(ch, (H.shape[1], 1)), "ewainit", max_iter=50)
    mx = bench.reduce_max(float(rank + 1), world)
    sm = bench.reduce_sum(float(B_PER_RANK), world)
    gathered = [None] * world
    dist.all_gather_object(gathered, (shot0, est.tolist(), iters.tolist()))
    if rank == 0:
        out.put((mx, sm, gathered))
    dist.destroy_process_group()


def test_two_rank_sharding_matches_single_process():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    mx, sm, gathered = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert mx == 2.0 and sm == 2.0 * B_PER_RANK
    offsets = [g[0] for g in gathered]
    assert offsets == [0, B_PER_RANK]  # disjoint, consecutive shot ranges

    import bench
    import oracle
    from oracle import codes

    H, _ = codes.build_code("planar", 5)
    ch = oracle.depolarizing(0.06)
    _, syn = oracle.sample(H, *ch, seed=bench.SEED, shot0=0, B=2 * B_PER_RANK)
    est, _, iters = oracle.decode(H, syn, np.tile(ch, (H.shape[1], 1)), "ewainit", max_iter=50)
    est_sharded = np.concatenate([np.array(g[1]) for g in gathered])
    iters_sharded = np.concatenate([np.array(g[2]) for g in gathered])
    assert (est_sharded == est).all() and (iters_sharded == iters).all()
