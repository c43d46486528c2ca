"""The benchmark's multi-GPU arithmetic on CPU ranks (gloo, world size 2): replicas are timed
independently and the job's rate is all ranks' tetrahedra over the slowest rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    total_ms, tets, value = bench.job_throughput(dist, 100.0 * (rank + 1), 1000 * (rank + 1), 2, device="cpu")
    out[rank] = (total_ms, tets, value)
    dist.destroy_process_group()


def test_replica_rate_uses_the_slowest_rank_and_all_tetrahedra():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        total_ms, tets, value = res[r]
        assert total_ms == 200.0 and tets == 3000.0
        assert abs(value - 3000 * 2 / 0.2 / 1e6) < 1e-12


def test_single_rank_rate():
    import bench
    assert bench.job_throughput(None, 500.0, 1000000, 5) == (500.0, 1000000.0, 10.0)


def test_replicas_draw_independent_clouds():
    """Rank r triangulates the workload generated with seed + r (no shared input)."""
    from paper_1805_08831_gb300 import synth
    a, b = synth.make("uniform", 1000, 2), synth.make("uniform", 1000, 3)
    assert a.shape == b.shape and not (a == b).all()


def test_cpu_paper_scheme_leg_reports_an_exact_rate():
    """The bench's second host baseline on a small sample: every host core, tetrahedra equal to
    the serial oracle's, and a rate computed from them."""
    import numpy as np

    import bench
    import oracle
    from paper_1805_08831_gb300 import synth
    x = synth.uniform_cube(20000, 2)
    ref, _ = oracle.delaunay(x, seed=bench.SEED)
    leg = bench.cpu_paper_scheme(x, ref)
    assert "error" not in leg, leg
    assert leg["bit_exact_vs_oracle"] is True and leg["cores"] == (os.cpu_count() or 1)
    assert leg["value"] > 0 and leg["unit"] == "Mtets/s" and leg["passes"] >= 3
    assert np.isfinite(leg["value"])
