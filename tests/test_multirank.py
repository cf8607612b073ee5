"""The N > 1 benchmark path on CPU: two gloo ranks (no GPU).

Replicas are independent (Sec. 3.1 uncertainty), so the GPUs shard them with
no data-path collective: each rank offsets the run seed, the timing is the
slowest rank's, and the value is every rank's units over that time.  Also
checks, with the oracle, that the two ranks' replica streams differ.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = 10.0 + 5.0 * rank                # rank 1 is the slow one
        ms_max = bench.max_over_ranks(ms_local, world, "cpu")
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.rank_seed(1002, rank))
        dist.barrier()
        value = bench.whole_job_rate(1000, world, 3, ms_max / 1e3)
        np.save(os.path.join(out_dir, f"r{rank}.npy"),
                np.array([ms_max, value, seeds[0], seeds[1]], dtype=np.float64))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_and_shard_seeds(tmp_path):
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r0 = np.load(tmp_path / "r0.npy")
    r1 = np.load(tmp_path / "r1.npy")
    assert r0[0] == r1[0] == 15.0                  # both ranks see the slowest time
    assert r0[1] == pytest.approx(1000 * 2 * 3 / 0.015)
    assert r0[2] == 1002 and r0[3] == 1002 + 7919 and r0[2] != r0[3]


def test_rank_seeds_give_different_replicas():
    import c2f_synth as S
    import oracle
    w = S.config2(side=40, n_replicas=4, hours=2)
    L = w.landscape
    p0 = dict(w.params, seed=bench.rank_seed(w.params["seed"], 0))
    p1 = dict(w.params, seed=bench.rank_seed(w.params["seed"], 1))
    o0 = oracle.Oracle(L.fuel, L.slope, L.aspect, cell_size=L.cell_size, weather=w.weather, **p0)
    o1 = oracle.Oracle(L.fuel, L.slope, L.aspect, cell_size=L.cell_size, weather=w.weather, **p1)
    cells0 = [o0.ignition_cell(r) for r in range(4)]
    cells1 = [o1.ignition_cell(r) for r in range(4)]
    assert cells0 != cells1
