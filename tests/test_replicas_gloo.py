"""The multi-GPU form is replicas: each rank builds its own graph, runs its own
sources, and the job's value is all ranks' traversed edges over the slowest
rank's time.  The rank logic runs here as two gloo processes on the CPU."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import bench
    import graphgen

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # per-rank inputs as the bench makes them: same graph seed, disjoint source draws
    w = dict(kind="rmat", scale=10, th=64, seed=10, src_seed=1001)
    src, dst = bench.make_edges_host(w)
    mask = graphgen.nonisolated_mask_host(1 << w["scale"], src, dst)
    sources = bench.sources_for(w, mask, rank)
    run_s = [0.5, 2.0][rank]
    wall_s = [3.0, 1.0][rank]
    edges = [1e9, 3e9][rank]
    value, run_max, wall_max = bench.replica_value(run_s, wall_s, edges, "cpu")
    out[rank] = (value, run_max, wall_max, sources.tolist())
    dist.barrier()
    dist.destroy_process_group()


def test_replica_value_two_gloo_ranks():
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    for r in (0, 1):
        value, run_max, wall_max, _ = out[r]
        assert run_max == 2.0 and wall_max == 3.0
        assert abs(value - (1e9 + 3e9) / 2.0 / 1e9) < 1e-12  # all edges / slowest rank
    s0, s1 = np.array(out[0][3]), np.array(out[1][3])
    assert len(s0) == len(s1) == 64
    assert not np.array_equal(s0, s1)  # each rank runs its own sources


def test_reference_arm_other_ranks_do_nothing(capsys):
    import bench

    class A:
        steps, warmup, workload = 1, 0, "rmat16"

    bench.run_reference(A(), bench.WORKLOADS["rmat16"], 2, 1)
    assert capsys.readouterr().out == ""
