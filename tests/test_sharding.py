"""Target-sharded evaluation on world_size-2 gloo CPU ranks: each rank owns a
contiguous range of stars, receives the full state by all-gather, computes its
stars' accelerations and its stars' part of the hole's sums (Eq. 1-3, with
the oracle as the per-rank engine); the hole's parts are summed by an
all-reduce, the stars' accelerations all-gathered.  The stars equal the
unsharded evaluation bit for bit, the hole within the rounding of the
reordered sum."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1801_07986_b300.shard import owner_of, shard_ranges


def test_shard_ranges_cover_every_star_once():
    for n in (2, 3, 257, 1000, 131072):
        for world in (1, 2, 3, 8):
            rs = shard_ranges(n, world)
            assert len(rs) == world
            covered = [b for a, e in rs for b in range(a, e)]
            assert covered == list(range(1, n))
            for a, e in rs[:-1]:
                assert (e - a) % 256 == 0 or e == n
            assert owner_of(0, rs) == 0
            assert all(a <= b for a, b in rs)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, n, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_1801_07986_b300.inputs import make_cluster
    x, v, m = make_cluster(n, 0.1, 7)
    rs = shard_ranges(n, world)
    a0, a1 = rs[rank]
    # each rank starts with only its own stars' state (plus the hole on rank 0)
    mine = torch.tensor(np.concatenate([x[a0:a1], v[a0:a1]], axis=1))
    sizes = [e - s for s, e in rs]
    cap = max(sizes)            # gloo all-gathers equal sizes: pad, then trim
    gathered = [torch.zeros((cap, 6), dtype=torch.float64) for _ in sizes]
    dist.all_gather(gathered, torch.nn.functional.pad(mine, (0, 0, 0, cap - mine.shape[0])))
    full = torch.cat([g[:sz] for g, sz in zip(gathered, sizes)]).numpy()
    xs = np.concatenate([x[:1], full[:, :3]])
    vs = np.concatenate([v[:1], full[:, 3:]])
    targets = np.arange(a0, a1)
    acc = oracle.accel_rows(xs, vs, m, targets, c=20.0, eps=1e-3) if a1 > a0 else np.zeros((0, 3))
    parts = [torch.zeros((cap, 3), dtype=torch.float64) for _ in sizes]
    dist.all_gather(parts, torch.nn.functional.pad(torch.tensor(acc), (0, 0, 0, cap - acc.shape[0])))
    parts = [p[:sz] for p, sz in zip(parts, sizes)]
    # the hole: this rank's outer stars' share of Eq. 1-3, summed over ranks
    if a1 > a0:
        newt, pn = oracle.bh_partial(xs, vs, m, a0, a1, eps=1e-3)
    else:
        newt, pn = np.zeros(3), np.zeros(3)
    red = torch.tensor(np.concatenate([newt, pn, np.abs(newt), np.abs(pn)]))
    dist.all_reduce(red, op=dist.ReduceOp.SUM)
    red = red.numpy()
    inv_c2 = 1.0 / (20.0 * 20.0)
    hole = red[:3] + inv_c2 * red[3:6]
    scale = red[6:9] + inv_c2 * red[9:12]
    if rank == 0:
        np.save(out_path, np.concatenate([hole[None], torch.cat(parts).numpy(), scale[None]]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_sharded_evaluation_equals_unsharded(tmp_path, world):
    import oracle
    from paper_1801_07986_b300.inputs import make_cluster
    n = 700
    out = str(tmp_path / "a.npy")
    mp.start_processes(_worker, args=(world, _free_port(), n, out), nprocs=world,
                       start_method="spawn")
    x, v, m = make_cluster(n, 0.1, 7)
    want = oracle.accel(x, v, m, c=20.0, eps=1e-3)
    got = np.load(out)
    scale = got[-1]
    got = got[:-1]
    assert np.array_equal(got[1:], want[1:])
    assert np.all(np.abs(got[0] - want[0]) <= 1e-14 * scale), (got[0], want[0])
