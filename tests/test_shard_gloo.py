"""The multi-rank path on CPU: local problems (Section 3) sharded over ranks with no data
exchange, and the bench's cross-rank timing reductions, as world-size-2 gloo process groups."""
import json
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1312_0195_gb300.shard import leaf_shard  # noqa: E402


@pytest.mark.parametrize("world", [1, 2, 3, 4, 7, 8])
def test_leaf_shard_tiles_the_list_and_balances_work(world):
    rng = np.random.default_rng(world)
    sizes = rng.choice([8, 16, 32, 64], size=997, p=[0.7, 0.15, 0.1, 0.05])
    ranges = [leaf_shard(sizes, r, world) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == len(sizes)
    for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
        assert a1 == b0 and a0 <= a1
    work = sizes.astype(np.int64) ** 2
    share = [int(work[a:b].sum()) for a, b in ranges]
    assert sum(share) == int(work.sum())
    assert max(abs(w - work.sum() / world) for w in share) <= work.max()


def test_leaf_shard_edge_cases():
    assert leaf_shard([], 0, 3) == (0, 0)
    assert [leaf_shard([8], r, 3) for r in range(3)] == [(0, 0), (0, 0), (0, 1)]
    with pytest.raises(ValueError):
        leaf_shard([8, 8], 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _field_and_leaves():
    import synth
    kap = synth.lognormal_kappa(64, 64, 4.0, 1.0, seed=21)
    leaves = synth.quadtree_leaves(64, 64, seed=22, root=32, min_size=4, p_split=0.7)
    leaves = leaves[leaves[:, 2] <= 8][:24]       # small leaves: the oracle solves each in milliseconds
    return kap, leaves


def _solve(kap, leaves):
    import oracle
    out = []
    for x0, y0, s in leaves:
        r = oracle.local_keff(kap[y0:y0 + s, x0:x0 + s], 1.0, 1.0 / 6.0, 1.0, 1e-6, tol=1e-8, max_steps=20000)
        out.append([float(v) for v in r["keff"]])
    return out


def _cubes():
    """3-D local problems as the bench shards them: equal cubes of a small log-normal box."""
    import synth
    k3 = synth.lognormal_kappa3d(8, 8, 8, 2.0, 1.0, seed=23)
    return k3, [(x, y, z, 4) for z in (0, 4) for y in (0, 4) for x in (0, 4)]


def _solve3(k3, cubes):
    import oracle
    out = []
    for x0, y0, z0, s in cubes:
        r = oracle.local_keff3(k3[z0:z0 + s, y0:y0 + s, x0:x0 + s].astype(np.float64), 1.0, 1.0 / 6.0, 1.0, 1e-6,
                               tol=1e-8, max_steps=20000)
        out.append([float(v) for v in r["keff"].ravel()])
    return out


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    ws, r, _ = bench.dist_init()
    assert (ws, r) == (world, rank) and dist.get_backend() == "gloo"
    kap, leaves = _field_and_leaves()
    lo, hi = leaf_shard(leaves[:, 2], rank, world)
    mine = _solve(kap, leaves[lo:hi])                    # no exchange while solving
    k3, cubes = _cubes()
    lo3, hi3 = leaf_shard(np.full(len(cubes), 4), rank, world)
    mine3 = _solve3(k3, cubes[lo3:hi3])
    bench.barrier(ws)
    t_max = bench.max_over_ranks(float(rank + 1), ws)
    n_sum = bench.sum_over_ranks(float(hi - lo), ws)
    gathered = [None] * world
    dist.all_gather_object(gathered, (lo, hi, mine, lo3, hi3, mine3))   # off the hot path: results to rank 0
    if rank == 0:
        with open(out_path, "w") as fh:
            json.dump({"t_max": t_max, "n_sum": n_sum, "parts": gathered}, fh)
    dist.destroy_process_group()


def test_two_gloo_ranks_solve_their_shards_like_one_process(tmp_path):
    import torch.multiprocessing as mp
    out = tmp_path / "gathered.json"
    mp.start_processes(_rank_main, args=(2, _free_port(), str(out)), nprocs=2, start_method="spawn", join=True)
    res = json.loads(out.read_text())
    kap, leaves = _field_and_leaves()
    assert res["t_max"] == 2.0 and res["n_sum"] == len(leaves)
    parts = sorted(res["parts"], key=lambda p: p[0])
    assert parts[0][0] == 0 and parts[-1][1] == len(leaves) and parts[0][1] == parts[1][0]
    sharded = [k for p in parts for k in p[2]]
    assert sharded == _solve(kap, leaves)                # bitwise: same problems, same arithmetic
    k3, cubes = _cubes()
    parts3 = sorted(((p[3], p[4], p[5]) for p in res["parts"]), key=lambda p: p[0])
    assert parts3[0][0] == 0 and parts3[-1][1] == len(cubes) and parts3[0][1] == parts3[1][0]
    assert [k for p in parts3 for k in p[2]] == _solve3(k3, cubes)
