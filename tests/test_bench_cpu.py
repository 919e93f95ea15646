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


def test_hbm_peak_prefers_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    v, src = bench.hbm_peak()
    assert v == 6800.0 and "fallback" in src
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 7000.5}))
    v, src = bench.hbm_peak()
    assert v == 7000.5 and "measured" in src


def test_walk_traffic_only_while_the_sources_match(tmp_path, monkeypatch):
    # a copy of the walk's sources with a profile line keyed by their hash
    src_dir = tmp_path / "paper_2009_01177_gb300" / "csrc"
    src_dir.mkdir(parents=True)
    for f in bench.WALK_SOURCES:
        with open(os.path.join(bench.ROOT, f), "rb") as fh:
            (tmp_path / f).write_bytes(fh.read())
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sha = bench.walk_sources_sha256()
    (tmp_path / "profiles" / "k_dfs_fp64_k32.md").write_text(
        f"traffic_bytes_per_launch = 1.25e11 (walk sources sha256 {sha})\n")
    assert bench.walk_traffic(32) == 1.25e11
    assert bench.walk_traffic(30) is None                          # no summary for that size
    with open(tmp_path / bench.WALK_SOURCES[0], "ab") as fh:       # any edit to the kernel's sources
        fh.write(b"\n// changed\n")
    assert bench.walk_traffic(32) is None


def test_committed_summary_matches_the_committed_sources():
    # the figure in the repository is for the sources in the repository
    assert bench.walk_traffic(32) is not None


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
