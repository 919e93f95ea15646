"""Host logic of bench.py (no GPU): the paper's FLOP model, the peak lookup, and the
traffic figure that is reported only while the walk's sources are unchanged."""
import json
import os
from math import comb

import pytest

import bench


def test_paper_flop_model_counts_one_solve_per_subset():
    # Sec. 7.1.2 (Eq. linflops): a complex HPD solve of size n = 2i costs 4/3 n^3 + n^2 - 4/3 n flops
    for k in (1, 3, 10, 32):
        direct = sum(comb(k, i) * (4 / 3 * (2 * i) ** 3 + (2 * i) ** 2 - 4 / 3 * (2 * i)) for i in range(1, k + 1))
        assert bench.paper_flops(k) == pytest.approx(direct, rel=1e-12)
    assert bench.paper_flops(1) == 12.0
    # closed form by the binomial moments sum C(N,i) i = N 2^(N-1), sum C(N,i) i^2 = N (N+1) 2^(N-2)
    # and sum C(N,i) i^3 = N^2 (N+3) 2^(N-3) (Eq. tflops summed over i)
    for n in (2, 7, 32, 50):
        closed = (32 / 3 * n * n * (n + 3) * 2.0 ** (n - 3) + 4 * n * (n + 1) * 2.0 ** (n - 2)
                  - 8 / 3 * n * 2.0 ** (n - 1))
        assert bench.paper_flops(n) == pytest.approx(closed, rel=1e-12)


def test_hbm_peak_prefers_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    v, src = bench.hbm_peak()
    assert v == 6800.0 and "fallback" in src
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 7000.5}))
    v, src = bench.hbm_peak()
    assert v == 7000.5 and "measured" in src


@pytest.mark.parametrize("kernel", sorted(bench.KERNEL_SOURCES))
def test_recorded_traffic_only_while_the_sources_match(tmp_path, monkeypatch, kernel):
    # a copy of the kernel's sources with a profile line keyed by their hash
    (tmp_path / "paper_2009_01177_gb300" / "csrc").mkdir(parents=True)
    for f in bench.KERNEL_SOURCES[kernel]:
        with open(os.path.join(bench.ROOT, f), "rb") as fh:
            (tmp_path / f).write_bytes(fh.read())
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sha = bench.sources_sha256(kernel)
    (tmp_path / "profiles" / f"{kernel}_k32.md").write_text(
        f"traffic_bytes_per_launch = 1.25e11 (sources sha256 {sha})\n")
    assert bench.recorded_traffic(kernel, 32) == 1.25e11
    assert bench.recorded_traffic(kernel, 30) is None                  # no summary for that size
    with open(tmp_path / bench.KERNEL_SOURCES[kernel][0], "ab") as fh:  # any edit to the kernel's sources
        fh.write(b"\n// changed\n")
    assert bench.recorded_traffic(kernel, 32) is None


def test_walk_operation_model():
    # the walk over r modes visits every non-empty subset once (one pivot each); per subset it
    # approaches 1 pivot, 1/2 coefficient set, 2 pivot rows and 7 Schur entries (Sum 2^-n-1 n(2n+1))
    for r in (1, 2, 5):
        p, c, rows, e, n = bench.walk_ops(r)
        assert n == 2 ** r and p == 2 ** r - 1
    assert bench.walk_ops(2)[1:4] == (1, 2, 3)       # one child with one mode: one 3-entry update
    p, c, rows, e, n = bench.walk_ops(32)
    assert abs(p / n - 1) < 1e-9 and abs(c / n - 0.5) < 1e-9
    assert abs(rows / n - 2) < 1e-6 and abs(e / n - 7) < 1e-6
    assert bench.fx256_macs_per_subset(32) == pytest.approx(60 * 29 + 18, rel=1e-6)


def test_dram_rate_of_the_walk(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.dram_rate(None, 291.7) is None
    d = bench.dram_rate(1.1757e11, 291.7)                 # 117.6 GB in 291.7 ms
    assert d["gbs"] == pytest.approx(403.05, rel=1e-3)
    assert d["frac_of_hbm"] == pytest.approx(403.05 / 6800.0, rel=1e-3) and "fallback" in d["peak_source"]


def _max_rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    out[rank] = bench.max_over_ranks([1.0 + rank, 5.0 - rank], world, "cpu")
    dist.destroy_process_group()


def test_step_time_is_the_max_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    assert bench.max_over_ranks([2.5, 3], 1, "cpu") == [2.5, 3.0]
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = 29700 + os.getpid() % 1000
        procs = [ctx.Process(target=_max_rank_main, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs)
        assert out[0] == out[1] == [2.0, 5.0]
