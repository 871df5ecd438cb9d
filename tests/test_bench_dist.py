"""The multi-process path of bench.py on CPU: two gloo ranks on 127.0.0.1.

bench.py runs one independent product per rank (replicas, weak scaling):
no data moves between ranks; the only collectives are the barrier around
the timed region and the max over ranks of the elapsed time.  These tests
run those helpers as two real processes, and check the per-rank inputs and
the whole-job rate formula."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    w, r, _ = bench.dist_setup(None)
    assert (w, r) == (world, rank)
    assert dist.get_backend() == "gloo"
    bench.barrier(w)
    # each rank reports its own elapsed time; all must see the slowest
    mx = bench.max_over_ranks(10.0 + 5.0 * rank, w)
    bench.barrier(w)
    A, _ = bench.rank_operands("spread", 16, r)
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), np.array([mx, A[0, 0], A.sum()]))
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_gloo_two_ranks(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    r0 = np.load(tmp_path / "rank0.npy")
    r1 = np.load(tmp_path / "rank1.npy")
    assert r0[0] == r1[0] == 15.0  # max over ranks of 10 and 15
    assert r0[2] != r1[2]          # the ranks multiply different problems


def test_rank_inputs_and_rate():
    sys.path.insert(0, ROOT)
    import bench
    from paper_1211_1581_gb300 import inputs
    A0, B0 = bench.rank_operands("spread", 32, 0)
    A, B = inputs.gemm_operands("spread", 32, 32, 32, seed=0, cfg=2)
    assert np.array_equal(A0, A) and np.array_equal(B0, B)
    A1, B1 = bench.rank_operands("spread", 32, 1)
    assert not np.array_equal(A0, A1) and not np.array_equal(B0, B1)
    # 2 ranks x 3 steps x 2e12 flops in 1 s (the slowest rank) = 12 TFLOP/s
    assert bench.aggregate_rate(2, 2e12, 3, 1000.0) == pytest.approx(12.0)
    assert bench.aggregate_rate(1, 2e12, 3, 1000.0) == pytest.approx(6.0)


def test_reference_arm_other_ranks_exit_quietly(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    bench.main()
    assert capsys.readouterr().out == ""
