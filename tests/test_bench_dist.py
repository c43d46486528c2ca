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


def test_path_bytes_are_the_tables_terms():
    """The bench's algorithmic bytes per inserted point: the hot-path table's formula with the
    paper's mean cavity (|C| = 20) and ball (|B| = 26) and two walk steps, worked by hand:
    walk 2 * 104 = 208; cavity 46 * 32 + (15 + 26) * 24 + 46 * 8 = 1472 + 984 + 368 = 2824;
    ball 26 * 32 + 26 * 4 + 20 * 4 + 46 * 4 = 832 + 104 + 80 + 184 = 1200."""
    import bench
    st = {"n_unique": 1000, "sum_cavity": 20000, "sum_ball": 26000, "sum_walk": 4000, "n_attempts": 2000}
    terms, cfb = bench.path_bytes(st)
    assert cfb["V"] == 15.0 and cfb["w"] == 2.0
    assert terms == {"walk": 208.0, "cavity": 2824.0, "ball": 1200.0}


def test_kernel_hash_ignores_comments_only(tmp_path, monkeypatch):
    """The bench reports a captured DRAM traffic only while the kernel's sources hash the same;
    a change of comments or blank lines keeps the hash, a change of code does not."""
    import shutil

    import bench
    src = os.path.join(bench.ROOT, "paper_1805_08831_gb300", "csrc")
    dst = tmp_path / "paper_1805_08831_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES:
        shutil.copy(os.path.join(src, f), dst / f)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_sources_hash()
    p = dst / "async.cu"
    text = p.read_text()
    p.write_text("// a new comment\n\n/* and a block\n   comment */\n" + text.replace("\n", "  // note\n", 3))
    assert bench.kernel_sources_hash() == h0
    p.write_text(text.replace("constexpr int kADefer = 16;", "constexpr int kADefer = 17;"))
    assert bench.kernel_sources_hash() != h0
