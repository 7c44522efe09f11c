"""The N > 1 host logic of bench.py on CPU with two gloo ranks: the batch's
cases are split over the ranks with nothing lost or duplicated and a
balanced load (longest-processing-time split), and the job's time is the
slowest rank's while its work is the sum of the ranks'."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    from paper_2406_07441_gb300 import cloudgen as cg
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        cases = cg.batch_cases()
        mine = bench._shard(cases, rank, world)
        allm = [None] * world
        dist.all_gather_object(allm, mine)
        load = sum(cases[k]["n_i"] * cases[k]["n_j"] for k in mine)
        ms, (work, ncase) = bench.combine_over_ranks(dist, 10.0 + 2.5 * rank, [float(load), float(len(mine))], "cpu")
        if rank == 0:
            q.put((allm, ms, work, ncase, sum(c["n_i"] * c["n_j"] for c in cases), len(cases),
                   [sum(cases[k]["n_i"] * cases[k]["n_j"] for k in m) for m in allm]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_batch_sharding_and_combining_over_gloo_ranks(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    allm, ms, work, ncase, total, ncases, loads = q.get(timeout=120)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    flat = sorted(k for m in allm for k in m)
    assert flat == list(range(ncases))                     # every case exactly once
    assert ms == 10.0 + 2.5 * (world - 1)                    # slowest rank
    assert work == total and ncase == ncases                 # summed work
    assert max(loads) <= 1.1 * min(loads)                    # balanced


def _rank_cloud(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import numpy as np

    import bench
    os.environ["TMPDIR"] = os.environ.get("LSKUM_TEST_TMP", "/tmp")
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        c = bench._shared_cloud("naca0012_160x64", rank, world, dist)
        h = [float(np.sum(c.x)), float(np.sum(c.y)), int(np.sum(c.nbr_idx)), int(c.nbr_off[-1]), int(c.n)]
        allh = [None] * world
        dist.all_gather_object(allh, h)
        if rank == 0:
            q.put(allh)
    finally:
        dist.destroy_process_group()


def test_ranks_share_one_cloud_built_on_rank_0(tmp_path):
    """With several ranks, rank 0 builds the workload's cloud once and the
    others load it from a temporary file: every rank holds the same arrays
    (and the file is gone afterwards)."""
    world = 2
    os.environ["LSKUM_TEST_TMP"] = str(tmp_path)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_cloud, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    allh = q.get(timeout=120)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert allh[0] == allh[1] and allh[0][4] == 10240
    assert not list(tmp_path.iterdir())
