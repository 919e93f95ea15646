#!/usr/bin/env python
"""Benchmark: subset determinants per second of the Torontonian on one click pattern.

Workload: the Torontonian of a k = 32 click pattern (64 x 64 FP64 matrix,
2^32 subsets) of a synthetic M = 100 mode lossy GBS state (r ~ U[0.6, 1.2],
Haar U, eta = 0.3, seed 2).  One step = one full Torontonian through the
library's AUTO path with tol = 1e-10: the FP32 bound pass routes the instance
to the tier that resolves it (the 256-bit-class fixed point at this kappa,
about 1e28), then prep (I - O, basis) + chunk roots + depth-first walk + exact
reduction, and the result's a-posteriori bound is checked against tol (the
run exits non-zero when it is missed).  The FP64 walk on the same instance is
reported beside it as a kernel-quality figure only: it does not resolve Tor.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
  python bench.py --mode batch   # 4096 click patterns, one scheduled batch vs one launch each
  python bench.py --mode mh      # MH sampling, learned vs plain proposal (M = 60; TV at M = 20)

Prints one JSON line on rank 0.  Under torchrun (N > 1) the ranks split the
chunks of the one Torontonian (Algorithm 1's rank partition) and add their
exact partial sums with one all-gather (strong scaling).

--impl reference times the CPU oracle (256-bit fixed-point direct subset
sum, test infrastructure) on a bounded sample of the same workload.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "subset-dets/s & % FP64 peak (k=32 Tor); batched Tor/s and accepted samples/s vs plain"
UNIT = "subset-dets/s"
# algorithmic FP64 flops per subset determinant (rank-2 Schur update amortised
# ~20 FMA = 40 flops, 2x2 det 3, rsqrt 1, product 1, accumulation 11)
FLOPS_PER_SUBSET = 55.0
# FP64 peak derived from unit counts and clocks: 2 DFMA/clk/SM x 152 SMs x 2.07 GHz x 2 flops
PEAK_TFLOPS = 2 * 152 * 2.07e9 * 2 / 1e12
L2_FLUSH_BYTES = 256 << 20


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def max_over_ranks(values, world, device):
    """Each value's maximum over the ranks of the default process group (the slowest rank's
    time sets a weak-scaling step); the values unchanged at world size 1."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def workload(k, rank):
    from paper_2009_01177_gb300 import gbs_inputs as gi
    st, pat, O = gi.workload_m100(k, seed=2, pattern_seed=None if rank == 0 else 2000 + rank)
    return st, pat, O


# sources whose compiled kernel a recorded ncu figure belongs to: a DRAM
# traffic figure is reported only while they are unchanged
_CSRC = "paper_2009_01177_gb300/csrc/"
KERNEL_SOURCES = {
    "k_dfs_fx9": [_CSRC + f for f in ("fx9.cuh", "tor_fx9.cuh", "fixacc.cuh", "tor_dfs.cuh", "tor_walk.cuh",
                                      "tor_kernels.cu", "tor_internal.h", "capi.cu")],
    "k_dfs_fp64": [_CSRC + f for f in ("tor_dfs.cuh", "tor_walk.cuh", "fixacc.cuh", "dd.cuh", "fx128.cuh",
                                       "tor_kernels.cu", "tor_internal.h", "capi.cu")],
}


def sources_sha256(kernel):
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def recorded_traffic(kernel, k):
    """DRAM bytes per launch of `kernel` at k from the committed ncu summary
    profiles/<kernel>_k<k>.md, if it was taken on the current sources."""
    import re
    path = os.path.join(ROOT, "profiles", f"{kernel}_k{k}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch = ([0-9.eE+]+) \(sources sha256 ([0-9a-f]{64})\)", text)
    if not m or m.group(2) != sources_sha256(kernel):
        return None
    return float(m.group(1))


TIER_NAME = {1: "fp64", 2: "dd", 3: "fx128", 4: "fx256"}
# the 256-bit-class tier's limb products: a product of two nine-limb values
# forms the limb pairs i + j >= 6, 60 signed 32 x 32 -> 64-bit multiply-adds
MAC_PER_PRODUCT = 60


def walk_ops(r):
    """Operations of the depth-first walk over the 2^r subsets of r modes (the prefix tree of
    Eq. 2's subsets, each child's Schur complement from its parent's): (pivot steps, pivot
    coefficient sets, pivot rows, Schur entries updated, subsets)."""
    import functools

    @functools.lru_cache(None)
    def node(m):
        p = c = rows = e = n = 0
        for cur in range(m):
            p += 1
            n += 1
            if cur > 0:
                c += 1
                rows += 2 * cur
                e += cur * (2 * cur + 1)
                a = node(cur)
                p, c, rows, e, n = p + a[0], c + a[1], rows + a[2], e + a[3], n + a[4]
        return p, c, rows, e, n

    p, c, rows, e, n = node(r)
    return p, c, rows, e, n + 1


# the reciprocal square root's one fixed-point Newton step ends in a product
# with an error term of four non-zero limbs: limb pairs i + j >= 6 with j <= 3
MAC_SHORT_PRODUCT = 18


def fx256_macs_per_subset(k):
    """Algorithmic limb multiply-adds per subset of the 256-bit-class walk: per subset its
    pivot (2x2 determinant: 2 products; the reciprocal square root from a double-double seed:
    y^2 and det2 y^2, then a short product; the term t y: 1), per non-leaf pivot the
    coefficients D^-1 (4), per pivot row the vector D^-1 u (4), per Schur entry the rank-2
    update (2); each full product 60 MACs, the short one 18."""
    p, c, rows, e, n = walk_ops(k)
    return (MAC_PER_PRODUCT * (5 * p + 4 * c + 4 * rows + 2 * e) + MAC_SHORT_PRODUCT * p) / n


def hbm_peak():
    """(GB/s, source): the measured copy bandwidth of this machine's GPUs when the measured-peaks
    file is present, else the recipe's fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            v = float(json.load(fh)["hbm_gbs"])
        return v, "of measured (copy bandwidth, MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, ValueError, KeyError, TypeError):
        return 6800.0, "of fallback (6.8 TB/s)"


def dram_rate(traffic, kernel_ms):
    """The kernel's measured DRAM traffic over its live-timed duration, against the HBM copy peak
    (the walk is not memory-bound; this shows by how far), or None without a traffic figure."""
    if traffic is None or not kernel_ms:
        return None
    peak, src = hbm_peak()
    gbs = traffic / (kernel_ms * 1e-3) / 1e9
    return {"gbs": gbs, "frac_of_hbm": gbs / peak, "hbm_peak_gbs": peak, "peak_source": src}


def paper_flops(k):
    """The paper's operation count for one Torontonian of k modes (Sec. 7.1.2, Eq. tflops): a
    Hermitian positive definite complex solve of size n = 2i, 4/3 n^3 + n^2 - 4/3 n flops
    (Eq. linflops), for each of the C(k, i) subsets of size i."""
    from math import comb
    return float(sum(comb(k, i) * (32 * i ** 3 + 12 * i ** 2 - 8 * i) / 3 for i in range(1, k + 1)))


DTYPE_OF = {"fp64": "f64", "dd": "f64x2 (double-double)", "fx128": "fixed128",
            "fx256": "fixed256 (nine 29-bit i32 limbs, 203 fraction bits)"}


def config(k, extra=None):
    c = {"workload": f"single Torontonian k={k} ({2 * k}x{2 * k} FP64 O_S) of a synthetic M=100 lossy "
                     f"GBS state (r~U[0.6,1.2], Haar U, eta=0.3, seed 2)",
         "k": k, "subsets_per_step": 2 ** k,
         "l2": "flushed between timed steps (256 MiB device write)"}
    if extra:
        c.update(extra)
    return c


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        try:
            with open(self.f.name) as fh:
                for line in fh:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                        rows.append(parts)
        finally:
            os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(float(r[2]) for r in rows)),
                "samples": len(rows), "reasons": reasons}


def cpu_oracle_sample(O, k, budget_s=15.0, chunk_log=8, seed=0, max_chunks=400):
    """Time the oracle on random 2^chunk_log-subset chunks of the same matrix."""
    import oracle
    rng = np.random.default_rng(seed)
    nchunks_total = 1 << (k - chunk_log)
    done, t0 = 0, time.perf_counter()
    while done < max_chunks:
        c = int(rng.integers(nchunks_total))
        oracle.tor_range(O, c << chunk_log, (c + 1) << chunk_log)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    return done << chunk_log, el, done


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    k = args.k
    st, pat, O = workload(k, 0)
    threads = os.cpu_count()
    per_step = []
    for i in range(args.warmup + args.steps):
        n, el, nch = cpu_oracle_sample(O, k, budget_s=1e9, chunk_log=8, seed=100 + i, max_chunks=4)
        if i >= args.warmup:
            per_step.append((n, el))
    subsets = sum(n for n, _ in per_step)
    secs = sum(e for _, e in per_step)
    value = subsets / secs
    sample = (f"each step: 4 random 256-subset chunks (masks [c 2^8, (c+1) 2^8)) of the k={k} matrix; "
              "256-bit fixed-point direct subset sum, OpenMP over masks")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / len(per_step),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "fixed256",
            "data": "synthetic", "config": config(k, {"tier": "oracle (256-bit fixed point, CPU)",
                                                     "l2": "not applicable (host cores)"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def marginals(st):
    """Exact single-mode click probabilities 1 - 1/sqrt(det Sigma_jj) (input side)."""
    import math
    M = st.M
    return np.array([1.0 - 1.0 / math.sqrt(np.linalg.det(st.Sigma[np.ix_([j, M + j], [j, M + j])]))
                     for j in range(M)])


def batch_patterns_m100(n, seed=4, k_lo=8, k_hi=30):
    """Click patterns of the M = 100 state: independent clicks with the exact
    single-mode marginals, kept when k_lo <= k <= k_hi (a stand-in for the
    chain-rule sampler's patterns; same state, same click-count range)."""
    from paper_2009_01177_gb300 import gbs_inputs as gi
    st = gi.lossy_gbs_state(100, 0.6, 1.2, 0.3, seed)
    marg = marginals(st)
    rng = np.random.default_rng(seed)
    pats = []
    while len(pats) < n:
        x = (rng.random(st.M) < marg).astype(np.uint8)
        if k_lo <= x.sum() <= k_hi:
            pats.append(x)
    return st, np.array(pats)


def run_adaptive(args):
    """Adaptive precision: the bound pass routes a k=40 instance of a brighter M=100 state,
    and timed random windows of chunks at the routed tier project the full k=40 and k=50 runs."""
    import math
    import torch
    from paper_2009_01177_gb300 import gbs_inputs as gi
    from paper_2009_01177_gb300 import tor
    ctx = tor.Context(0)
    st = gi.lossy_gbs_state(100, 0.8, 1.4, 0.3, 3)
    pat = gi.random_pattern(100, 50, 1003)
    tol = 1e-10
    rng = np.random.default_rng(3)
    # walked modes per chunk: at k >= 40 a chunk's root eliminates 23+ modes, so
    # longer chunks than the k <= 32 defaults keep the root a few percent of the walk
    r1_of = {"fp64": 16, "dd": 13, "fx128": 13, "fx256": 17}
    # each window is whole waves of the resident grid (3 blocks of 128 threads per SM, the
    # tuned k = 32 launch of every tier), so no partial last wave skews the rate
    bps, tpb = 3, 128
    ctx.set_launch(tpb, bps)
    threads = torch.cuda.get_device_properties(0).multi_processor_count * bps * tpb
    waves_of = {"fp64": 4, "dd": 4, "fx128": 4, "fx256": 2}
    window_of = {p: w * threads for p, w in waves_of.items()}
    out = {"metric": "adaptive precision: routed tier and projected single-GPU runtime (k=40, k=50)",
           "unit": "subset-dets/s", "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
           "config": {"workload": "M=100 synthetic lossy GBS state (r~U[0.8,1.4], Haar U, eta=0.3, seed 3), "
                                  "nested random patterns of k=40 and k=50 clicks; tol=1e-10",
                      "window_chunks": window_of, "window_waves": waves_of,
                      "launch": {"threads_per_block": tpb, "blocks_per_sm": bps},
                      "l2": "inputs resident (the walk reads a 2k x 2k matrix)"}}
    with ClockSampler(0) as clocks:
        for k in (40, 50):
            Od = torch.from_numpy(gi.select(st.O, pat[:k])).cuda()
            bd = ctx.bounds([Od], tol=tol)[0]
            routed = {1: "fp64", 2: "dd", 3: "fx128", 4: "fx256"}[int(bd["tier"])]
            rows = {}
            for prec in dict.fromkeys([routed, "fp64"]):
                d = k - r1_of[prec]
                window = window_of[prec]
                nchunks = 1 << d
                ms = []
                for w in range(4):
                    c0 = int(rng.integers(0, nchunks - window + 1))
                    if w == 0:                # warm-up window, not timed
                        ctx.chunks(Od, d, c0, c0 + window, prec=prec)
                        torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    ctx.chunks(Od, d, c0, c0 + window, prec=prec)
                    e1.record()
                    torch.cuda.synchronize()
                    ms.append(e0.elapsed_time(e1))
                mean = float(np.mean(ms))
                rate = window * (1 << (k - d)) / (mean * 1e-3)
                rows[prec] = {"chunk_bits": d, "windows_ms": [round(x, 2) for x in ms],
                              "window_cv": float(np.std(ms) / mean), "subset_dets_per_s": rate,
                              "projected_full_s": float(2.0 ** k / rate),
                              "paper_equivalent_tflops": paper_flops(k) / (2.0 ** k / rate) / 1e12}
            out[f"k{k}"] = {"routed_tier": routed, "bits_needed": bd["bits_needed"],
                            "log2_tmax": bd["log_tmax"] / math.log(2),
                            "log2_kappa_est": bd["log_kappa_est"] / math.log(2), "tiers": rows}
    if args.full_k40:            # the whole k = 40 Torontonian through the AUTO path, timed and checked
        Od = torch.from_numpy(gi.select(st.O, pat[:40])).cuda()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = ctx.single(Od, prec="auto", tol=tol)
        e1.record()
        torch.cuda.synchronize()
        s_full = e0.elapsed_time(e1) / 1e3
        out["k40_full"] = {"s": s_full, "subset_dets_per_s": 2.0 ** 40 / s_full, "tier": TIER_NAME[r.tier],
                           "tor": r.value, "hi": r.hi, "lo": r.lo, "sum_abs": r.sum_abs, "err_est": r.err_est,
                           "err_est_over_tor": r.err_est / abs(r.value), "kappa": r.kappa,
                           "resolved": bool(r.status == 0 and r.err_est <= tol * abs(r.value))}
    out["value"] = out["k40"]["tiers"][out["k40"]["routed_tier"]]["subset_dets_per_s"]
    out["dtype"] = out["k40"]["routed_tier"]
    out["clocks"] = clocks.summary()
    out["paper_context"] = "one k=50 Torontonian: 73,773 s (128-bit) and 170,891 s (256-bit) on 39,286 Sunway TaihuLight nodes"
    print(json.dumps(out), flush=True)
    ctx.close()


def run_table(args):
    """Every click pattern's Torontonian of one M-mode state (tor_all_patterns): one walk over
    the 2^M subsets and a Moebius transform, against the patterns one by one."""
    import math
    import torch
    from paper_2009_01177_gb300 import gbs_inputs as gi
    from paper_2009_01177_gb300 import tor
    ctx = tor.Context(0)
    M = args.table_m
    st = gi.lossy_gbs_state(M, 0.5, 1.0, 0.5, 5)
    Od = torch.from_numpy(st.O).cuda()
    s_, ld_ = np.linalg.slogdet(np.eye(2 * M) - st.O)
    prec = "fx128" if -0.5 * ld_ / math.log(2) <= 11 else "dd"
    n = 1 << M
    out = torch.zeros(n * tor.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        ctx.all_patterns_async(Od, out, prec=prec)
    torch.cuda.synchronize()
    ctx.set_timing(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    walk_ms, tr_ms = [], []
    with ClockSampler(0) as clocks:
        torch.cuda.synchronize()
        for i in range(args.steps):
            ev[i][0].record()
            ctx.all_patterns_async(Od, out, prec=prec)
            ev[i][1].record()
            walk_ms.append(ctx.walk_time_ms())
            tr_ms.append(ctx.transform_time_ms())
        torch.cuda.synchronize()
    ctx.set_timing(False)
    step_ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    walk = float(np.mean(walk_ms))
    tr = float(np.mean(tr_ms))
    # transform traffic per entry: the first pass reads the 32-byte term and writes it and its
    # 8-byte sum; every later pass reads and writes both; passes of 10 bits, then 5, the last shorter
    passes, b = 0, 0
    while b < M:
        b += 10 if b == 0 else 5
        passes += 1
    tr_bytes = n * (72 + (passes - 1) * 80) if M >= 10 else None
    # the patterns one by one (tor_batch_patterns), timed on a uniform sample and scaled to 2^M
    rng = np.random.default_rng(5)
    sample = (rng.random((4096, M)) < 0.5).astype(np.uint8)
    P = tor.pack_patterns(sample, M).cuda()
    ob = torch.zeros(4096 * tor.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    ctx.batch_patterns_async(Od, P, ob, prec=prec)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    ctx.batch_patterns_async(Od, P, ob, prec=prec)
    e1.record()
    torch.cuda.synchronize()
    per_pattern_s = e0.elapsed_time(e1) * 1e-3 / 4096
    r = tor.results_array(out, n)
    scale = math.exp(-0.5 * float(np.linalg.slogdet(st.Sigma)[1]))
    peak, peak_src = hbm_peak()
    line = {"metric": f"all 2^{M} click-pattern Torontonians of one state", "value": n / (step_ms * 1e-3),
            "unit": "Tor/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
            "higher_is_better": True, "dtype": prec, "data": "synthetic",
            "config": {"workload": f"M={M} synthetic lossy GBS state (r~U[0.5,1.0], Haar U, eta=0.5, seed 5); "
                                   f"tor_all_patterns: walk over 2^{M} subsets, Moebius transform of the exact "
                                   "term table", "l2": f"table of {n * 40 / 2**30:.2f} GiB, far above L2"},
            "walk_ms": walk, "walk_subset_dets_per_s": n / (walk * 1e-3), "transform_ms": tr,
            "roofline": {"bound": "hbm", "kernel": "k_mobius_pass (+ sums init)",
                         "achieved": tr_bytes / (tr * 1e-3) / 1e9 if tr_bytes else None,
                         "peak": peak, "unit": "GB/s",
                         "frac": tr_bytes / (tr * 1e-3) / 1e9 / peak if tr_bytes else None,
                         "traffic": None, "passes": passes, "peak_source": peak_src},
            "one_by_one": {"s_per_pattern": per_pattern_s, "projected_s": per_pattern_s * n,
                           "speedup": per_pattern_s * n / (step_ms * 1e-3),
                           "sample": "4096 uniform random patterns through tor_batch_patterns, same tier"},
            "sum_p": float((r["hi"] + r["lo"]).sum()) * scale, "statuses_ok": int((r["status"] == 0).sum()),
            "clocks": clocks.summary()}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_levels(args):
    """The prefix-tree walk against the paper's own schedule (a fresh elimination per subset,
    level by level) on the same GPU, same tier, same instance."""
    import torch
    from paper_2009_01177_gb300 import gbs_inputs as gi
    from paper_2009_01177_gb300 import tor
    ctx = tor.Context(0)
    st, pat, O32 = gi.workload_m100(32)
    rows = {}
    for k in (20, 24, 26):
        Od = torch.from_numpy(gi.select(st.O, pat[:k])).cuda()
        ctx.autotune(k, "fp64")
        for name, fn in (("walk", lambda: ctx.single(Od, prec="fp64")),
                         ("levels", lambda: tor.levels(Od, prec="fp64"))):
            r = fn()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                r = fn()
            torch.cuda.synchronize()
            el = (time.perf_counter() - t0) / args.steps
            rows.setdefault(f"k{k}", {})[name] = {"s": el, "subset_dets_per_s": 2.0 ** k / el, "tor": r.value,
                                                  "err_est": r.err_est}
        rows[f"k{k}"]["speedup_walk"] = rows[f"k{k}"]["levels"]["s"] / rows[f"k{k}"]["walk"]["s"]
    line = {"metric": "prefix-tree walk vs the paper's level schedule (fresh elimination per subset)",
            "value": rows["k26"]["speedup_walk"], "unit": "x", "n_gpus": 1, "higher_is_better": True,
            "dtype": "f64", "data": "synthetic", "steps": args.steps,
            "config": {"workload": "k = 20, 24, 26 patterns of the synthetic M=100 state (seed 2), FP64, "
                                   "tor_single (autotuned) against tor_levels, wall time per call"},
            "rows": rows}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_batch(args):
    """Batched Tor/s for 4096 patterns (k in [8, 30]) at tol, against the same Torontonians
    one launch each at the tier the batch settled on (equal accuracy)."""
    import torch
    from paper_2009_01177_gb300 import gbs_inputs as gi
    from paper_2009_01177_gb300 import tor
    tol = args.tol
    st, pats = batch_patterns_m100(args.n)
    ctx = tor.Context(0)
    sampler = None
    if args.patterns == "chainrule":   # exact chain-rule samples of the same state instead
        from paper_2009_01177_gb300 import chainrule
        stats = {}
        t0 = time.perf_counter()
        pats = chainrule.sample(ctx, st.Sigma, args.n, seed=4, k_min=8, k_max=30, prec="auto",
                                tol=args.mh_tol, form="noclick", stats=stats)
        torch.cuda.synchronize()
        sampler = {"s": time.perf_counter() - t0, "torontonians": stats["torontonians"],
                   "subsets": stats["subsets"], "tol": args.mh_tol,
                   "form": "no-click prefix probabilities, AUTO tiers, one tor_batch_patterns per mode"}
    ks = pats.sum(1)
    subsets = float((2.0 ** ks).sum())
    Od = torch.from_numpy(st.O).cuda()
    P = tor.pack_patterns(pats, st.M).cuda()
    n = len(pats)
    out = torch.zeros(n * tor.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    warm = tor.pack_patterns(pats[:64], st.M).cuda()
    for _ in range(args.warmup):              # warm-up on a 64-pattern slice of the same batch
        ctx.batch_patterns_async(Od, warm, out, prec="auto", tol=tol)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clocks:
        e0.record()
        for _ in range(args.steps):
            ctx.batch_patterns_async(Od, P, out, prec="auto", tol=tol)
        e1.record()
        torch.cuda.synchronize()
    tb = e0.elapsed_time(e1) / 1e3 / args.steps
    res = tor.results_from_tensor(out, n)
    tiers = [TIER_NAME.get(r.tier, "none") for r in res]
    ok = [r.status == 0 and r.err_est <= tol * abs(r.value) for r in res]
    ratio = [r.err_est / abs(r.value) if r.value else float("inf") for r in res]
    # the same Torontonians, one tor_single_async launch each at the batch's final tier
    mats = [torch.from_numpy(gi.select(st.O, np.nonzero(x)[0])).cuda() for x in pats]
    o1 = torch.zeros(n * tor.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    ctx.single_async(mats[0], o1[:tor.RESULT_BYTES], prec=tiers[0] if tiers[0] != "none" else "fp64")
    torch.cuda.synchronize()
    e0.record()
    for i, m in enumerate(mats):
        if tiers[i] != "none":
            ctx.single_async(m, o1[i * tor.RESULT_BYTES:(i + 1) * tor.RESULT_BYTES], prec=tiers[i])
    e1.record()
    torch.cuda.synchronize()
    ts = e0.elapsed_time(e1) / 1e3
    res1 = tor.results_from_tensor(o1, n)
    agree = sum(abs(a.value - b.value) <= a.err_est + b.err_est for a, b, t in zip(res, res1, tiers) if t != "none")
    line = {"metric": f"batched Tor/s ({n} patterns, k in [8,30]) at tol", "value": n / tb, "unit": "Tor/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tb,
            "higher_is_better": True, "dtype": "auto: " + ", ".join(sorted(set(tiers))), "data": "synthetic",
            "config": {"workload": f"{n} click patterns of a synthetic M=100 lossy GBS state "
                                   "(r~U[0.6,1.2], eta=0.3, seed 4): " +
                                   ("exact chain-rule samples of p(S | 8 <= k <= 30)" if sampler else
                                    "independent clicks with the exact single-mode marginals, kept if "
                                    "8 <= k <= 30"), "k_mean": float(ks.mean()),
                       "subsets": subsets, "prec": "auto", "tol": tol,
                       "warmup": "on a 64-pattern slice of the batch"},
            "subset_dets_per_s": subsets / tb,
            "tiers": {t: tiers.count(t) for t in sorted(set(tiers))},
            "resolved": int(sum(ok)), "eprec": int(sum(r.status == tor.TOR_EPREC for r in res)),
            "max_err_est_over_tor": float(max(ratio)),
            "one_launch_each": {"Tor/s": n / ts, "subset_dets_per_s": subsets / ts, "s": ts,
                                "tiers": "each instance at the batch's final tier",
                                "agree_within_bounds": int(agree)},
            "speedup_vs_one_launch_each": ts / tb,
            "clocks": clocks.summary()}
    if sampler:
        line["chain_rule_sampler"] = sampler
    print(json.dumps(line), flush=True)
    ctx.close()


def _click_counts(pat):
    """Click count of each row of an int64 (C, words) bitset tensor."""
    a = pat.cpu().numpy().view(np.uint8)
    return np.unpackbits(a, axis=1).sum(1)


def _ess_geyer(x):
    """Mean over chains of the effective sample size of a (T, C) series (Geyer's
    initial positive sequence estimator)."""
    T, C = x.shape
    x = x - x.mean(0)
    var = (x * x).mean(0) + 1e-12
    rho = np.stack([(x[:T - t] * x[t:]).mean(0) / var for t in range(T)])  # lags 0..T-1
    tau = np.ones(C)
    alive = np.ones(C, dtype=bool)
    for t in range(1, T - 1, 2):
        g = rho[t] + rho[t + 1]
        alive &= g > 0
        tau += np.where(alive, 2.0 * g, 0.0)
    return float(np.mean(T / np.maximum(tau, 1.0)))


def run_mh(args):
    """Accepted samples/s and ESS/s, learned vs plain proposal, same chains and tier;
    TV distance to all 2^20 exact probabilities at M = 20."""
    import math
    import torch
    from paper_2009_01177_gb300 import gbs_inputs as gi
    from paper_2009_01177_gb300 import tor
    ctx = tor.Context(0)
    C = args.n
    t_start = time.perf_counter()

    def progress(msg):
        print(f"[mh {time.perf_counter() - t_start:7.1f} s] {msg}", file=sys.stderr, flush=True)

    def chains(st, C=C):
        words = (st.M + 63) // 64
        return dict(O=torch.from_numpy(st.O).cuda(), logdet=float(np.linalg.slogdet(st.Sigma)[1]),
                    pat=torch.zeros((C, words), dtype=torch.int64, device="cuda"),
                    logp=torch.full((C,), -math.inf, dtype=torch.float64, device="cuda"),
                    logq=torch.zeros(C, dtype=torch.float64, device="cuda"),
                    acc=torch.zeros(C, dtype=torch.int32, device="cuda"), C=C,
                    marg=torch.tensor(marginals(st), dtype=torch.float64, device="cuda"))

    tol = args.mh_tol
    causes = {}   # rejections that were not the Metropolis test, by cause, per run label

    def run(ch, steps, seed, prop=None, record=None, t0=0, k_cap=0, label=None):
        """steps MH steps; the mean acceptance.  Every Torontonian comes from the AUTO path at
        tol; rejections for other reasons than the Metropolis test are counted by cause."""
        acc = torch.zeros((), dtype=torch.float64, device="cuda")
        cnt = torch.zeros(3, dtype=torch.int64, device="cuda")
        for s_ in range(steps):
            ctx.sample_step(ch["O"], ch["logdet"], ch["pat"], ch["logp"], ch["logq"], ch["acc"], seed, t0 + s_,
                            marg_p=ch["marg"], proposal=prop, prec="auto", tol=tol, k_cap=k_cap)
            a = ch["acc"]
            acc += (a == 1).double().mean()
            cnt += torch.stack([(a == -1).sum(), (a == -2).sum(), (a == -3).sum()])
            if record is not None:
                record.append(ch["pat"].clone())
        if label is not None:
            c = cnt.tolist()
            causes[label] = {"over_k_cap": c[0], "missed_tol": c[1], "failed": c[2], "proposals": steps * ch["C"]}
        return float(acc) / steps

    def run_da(ch, steps, seed, net, record=None, t0=0, k_cap=0, label=None):
        """steps delayed-acceptance steps (plain proposals screened by the network's density,
        the exact Torontonian only for the survivors); the mean acceptance."""
        if "logs" not in ch:          # the surrogate's log density of the current states
            ch["logs"] = net.logq(ch["pat"])
        acc = torch.zeros((), dtype=torch.float64, device="cuda")
        cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
        for s_ in range(steps):
            ctx.sample_step_da(ch["O"], ch["logdet"], ch["pat"], ch["logp"], ch["logq"], ch["logs"], ch["acc"], seed,
                               t0 + s_, marg_p=ch["marg"], surrogate=net, prec="auto", tol=tol, k_cap=k_cap)
            a = ch["acc"]
            acc += (a == 1).double().mean()
            cnt += torch.stack([(a == -1).sum(), (a == -2).sum(), (a == -3).sum(), (a == -4).sum()])
            if record is not None:
                record.append(ch["pat"].clone())
        if label is not None:
            c = cnt.tolist()
            causes[label] = {"over_k_cap": c[0], "missed_tol": c[1], "failed": c[2], "screened_out": c[3],
                             "proposals": steps * ch["C"]}
        return float(acc) / steps

    def train(net, pats, w, iters, batch, lr, val=None, val_w=None, resample=False):
        """Adam on the weighted NLL; with val, keep the parameters of best validation NLL
        (weighted by val_w when given).  resample: draw each batch with probability
        proportional to w and unit weights (the same expected gradient, less variance
        when the weights are heavy-tailed)."""
        best, best_theta, nll0 = None, None, None

        def val_nll():
            lq = net.logq(val)
            return float(-(lq * val_w).sum() / val_w.sum()) if val_w is not None else float(-lq.mean())
        if val is not None:
            nll0 = best = val_nll()
            best_theta = net.get_params(0)
        ones = torch.ones(batch, dtype=torch.float32, device="cuda")
        for it in range(iters):
            if resample:
                idx = torch.multinomial(w, batch, replacement=True)
                net.train_step(pats[idx].contiguous(), ones, lr=lr)
            else:
                idx = torch.randint(0, pats.shape[0], (batch,), device="cuda")
                net.train_step(pats[idx].contiguous(), w[idx].contiguous(), lr=lr)
            if val is not None and (it + 1) % 200 == 0:
                v = val_nll()
                if v < best:
                    best, best_theta = v, net.get_params(0)
        if val is not None:
            net.set_params(best_theta)
        return nll0, best

    # M = 60: train on states of the plain exact chain, then race the two proposals
    st = gi.lossy_gbs_state(60, 0.5, 1.0, 0.5, 6)
    marg60 = marginals(st)
    # the cost of one proposal is 2^k subset determinants: both chains target p(S | k <= k_cap)
    k_cap = int(round(marg60.sum() + 3.5 * np.sqrt((marg60 * (1 - marg60)).sum())))
    ch = chains(st)
    hist = []
    progress(f"M=60 plain exact chain, k_cap={k_cap}")
    run(ch, 60, 6, record=hist, k_cap=k_cap, label="training_chain")
    progress("training the proposal")
    pool = torch.cat(hist[10:])
    pool = pool[torch.randperm(pool.shape[0], device="cuda")]
    nval = pool.shape[0] // 10
    val, trn = pool[:nval].contiguous(), pool[nval:].contiguous()
    net = tor.MLP(ctx, st.M, 256, seed=6)
    net.set_marginals(marg60)                 # start at the plain proposal
    nll_plain, nll_learned = train(net, trn, torch.ones(trn.shape[0], dtype=torch.float32, device="cuda"),
                                   3000, 4096, 3e-4, val=val)
    # the same network trained instead on importance-weighted pairs the exact kernel scored:
    # proposals of the plain product proposal with weights p(S)/q(S), self-normalised
    progress("importance-weighted pairs")
    rng = np.random.default_rng(61)
    X = (rng.random((48 * C, st.M)) < marg60).astype(np.uint8)
    X = X[X.sum(1) <= k_cap]
    O60 = torch.from_numpy(st.O).cuda()
    Pis = tor.pack_patterns(X, st.M).cuda()
    ois = torch.zeros(X.shape[0] * tor.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    t_is = time.perf_counter()
    ctx.batch_patterns_async(O60, Pis, ois, prec="auto", tol=tol)
    torch.cuda.synchronize()
    t_is = time.perf_counter() - t_is
    ris = tor.results_array(ois, X.shape[0])
    tor_v = ris["hi"] + ris["lo"]
    ok = (ris["status"] == 0) & (tor_v > 0) & (ris["err_est"] <= tol * np.abs(tor_v))
    logdet60 = float(np.linalg.slogdet(st.Sigma)[1])
    logp_is = np.log(np.where(ok, tor_v, 1.0)) - 0.5 * logdet60
    logq_is = (X * np.log(marg60) + (1 - X) * np.log1p(-marg60)).sum(1)
    lw = np.where(ok, logp_is - logq_is, -np.inf)
    w_is = np.exp(lw - lw.max())
    w_is /= w_is.sum()
    ess_is = float(1.0 / (w_is ** 2).sum())
    perm = rng.permutation(X.shape[0])
    nv = X.shape[0] // 10
    wt = torch.tensor(w_is, dtype=torch.float32, device="cuda")
    vi, ti = torch.from_numpy(perm[:nv]).cuda(), torch.from_numpy(perm[nv:]).cuda()
    net_is = tor.MLP(ctx, st.M, 256, seed=6)
    net_is.set_marginals(marg60)
    progress(f"training on {X.shape[0]} weighted pairs (weight ESS {ess_is:.0f})")
    nll_is0, nll_is = train(net_is, Pis[ti].contiguous(), wt[ti].contiguous(), 3000, 4096, 3e-4,
                            val=Pis[vi].contiguous(), val_w=wt[vi].double().contiguous(), resample=True)
    res = {}
    steps = max(8, 4 * args.steps)
    for name, prop in (("plain", None), ("learned", net), ("learned_is", net_is), ("delayed_acceptance", net),
                       ("delayed_acceptance_is", net_is)):
        progress(f"race: {name}")
        chn = chains(st)
        step_fn = (lambda *a, **kw: run_da(*a[:3], a[3], *a[4:], **kw)) if name.startswith("delayed") else run
        step_fn(chn, 3, 7, prop, k_cap=k_cap)
        series = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        acc = step_fn(chn, steps, 7, prop, record=series, t0=100, k_cap=k_cap, label=name)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        ess = _ess_geyer(np.stack([_click_counts(p) for p in series]).astype(float))
        res[name] = {"acceptance": acc, "accepted_samples_per_s": acc * C * steps / el,
                     "ess_per_s": ess * C / el, "ess_per_chain": ess, "s": el, "steps": steps}
    out = {"metric": "accepted samples/s, learned vs plain proposal (M=60)", "unit": "samples/s",
           "value": res["learned"]["accepted_samples_per_s"], "n_gpus": 1, "higher_is_better": True,
           "dtype": "Torontonians by the AUTO path at tol (tiers as the bound pass routes), bf16 network",
           "data": "synthetic", "tol": tol, "rejections_not_by_the_test": causes, "plain": res["plain"],
           "learned": res["learned"],
           "speedup_accepted": res["learned"]["accepted_samples_per_s"] / res["plain"]["accepted_samples_per_s"],
           "speedup_ess": res["learned"]["ess_per_s"] / max(res["plain"]["ess_per_s"], 1e-30),
           "delayed_acceptance": dict(res["delayed_acceptance"], note="plain proposals screened by the "
                                      "learned network's density; exact Torontonians only for the survivors"),
           "speedup_ess_delayed_acceptance": res["delayed_acceptance"]["ess_per_s"] / max(res["plain"]["ess_per_s"],
                                                                                          1e-30),
           "speedup_accepted_delayed_acceptance": res["delayed_acceptance"]["accepted_samples_per_s"] /
                                                  res["plain"]["accepted_samples_per_s"],
           "delayed_acceptance_is": dict(res["delayed_acceptance_is"], note="the same, screened by the network "
                                         "trained on importance-weighted exact pairs"),
           "speedup_ess_delayed_acceptance_is": res["delayed_acceptance_is"]["ess_per_s"] /
                                                max(res["plain"]["ess_per_s"], 1e-30),
           "validation_nll": {"plain_proposal": nll_plain, "learned": nll_learned},
           "importance_weighted": {"pairs": int(X.shape[0]), "weight_ess": ess_is, "scoring_s": t_is,
                                   "weighted_validation_nll": {"plain_proposal": nll_is0, "learned_is": nll_is},
                                   "race": res["learned_is"],
                                   "speedup_accepted": res["learned_is"]["accepted_samples_per_s"] /
                                                       res["plain"]["accepted_samples_per_s"]},
           "k_cap": k_cap,
           "mean_clicks": float(marg60.sum()),
           "config": {"workload": f"M=60 synthetic lossy GBS state (r~U[0.5,1.0], eta=0.5, seed 6), {C} "
                                  "independence-MH chains targeting p(S | k <= k_cap); MADE 60-256-256-256-60 started at the "
                                  "plain proposal, trained (3000 Adam steps, batch 4096, best of held-out NLL) on "
                                  "50 x C states of the plain exact chain ('learned'), or on 48 x C proposals "
                                  "of the plain proposal scored by the exact kernel with self-normalised "
                                  "weights p/q ('learned_is')"}}
    # M = 20: all 2^20 exact probabilities, then TV of the pooled chain states
    progress("M=20 exact table")
    st20 = gi.lossy_gbs_state(20, 0.5, 1.0, 0.5, 5)
    allx = ((np.arange(1 << 20)[:, None] >> np.arange(20)[None, :]) & 1).astype(np.uint8)
    O20 = torch.from_numpy(st20.O).cuda()
    P20 = tor.pack_patterns(allx, 20).cuda()
    # every pattern's exact probability from one walk over the 2^20 subsets (tor_all_patterns)
    o20 = torch.zeros((1 << 20) * tor.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    ctx.all_patterns_async(O20, o20, prec="fx128")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.all_patterns_async(O20, o20, prec="fx128")
    torch.cuda.synchronize()
    t_exact = time.perf_counter() - t0
    r20 = tor.results_array(o20, 1 << 20)
    p20 = (r20["hi"] + r20["lo"]) * math.exp(-0.5 * np.linalg.slogdet(st20.Sigma)[1])
    net20 = tor.MLP(ctx, 20, 256, seed=5)
    net20.set_marginals(marginals(st20))
    train(net20, P20, torch.tensor(np.maximum(p20, 0), dtype=torch.float32, device="cuda"), 1500, 8192, 1e-3)
    tv, curve = {}, {}
    C20 = 16 * C
    checkpoints = (10, 25, 50, 100)
    for name, prop in (("plain", None), ("learned", net20)):
        progress(f"M=20 chains: {name}")
        chn = chains(st20, C20)
        run(chn, 20, 9, prop)
        series, pts, el = [], [], 0.0
        done = 0
        for cp in checkpoints:              # time only the steps; TV of all states pooled so far
            torch.cuda.synchronize()
            t0s = time.perf_counter()
            run(chn, cp - done, 9, prop, record=series, t0=20 + done, label=f"m20_{name}")
            torch.cuda.synchronize()
            el += time.perf_counter() - t0s
            done = cp
            codes = np.concatenate([p[:, 0].cpu().numpy() for p in series])
            freq = np.bincount(codes, minlength=1 << 20) / codes.size
            pts.append({"steps": cp, "s": el, "tv": 0.5 * float(np.abs(freq - p20).sum())})
        tv[name] = pts[-1]["tv"]
        curve[name] = pts
    out["m20"] = {"tv_pooled_100_steps": tv, "tv_vs_time": curve, "chains": C20, "samples_pooled": 100 * C20,
                  "exact_table_s": t_exact, "exact_table": "tor_all_patterns, 128-bit fixed point",
                  "sum_p": float(p20.sum()), "subset_dets": 2 ** 20,
                  "statuses_ok": int((r20["status"] == 0).sum())}
    print(json.dumps(out), flush=True)
    ctx.close()


def _timed_walks(ctx, Od, prec, reps):
    """Walk-kernel milliseconds of `reps` single_async calls at an explicit tier, and the last result."""
    import torch
    from paper_2009_01177_gb300 import tor
    out = torch.empty(tor.RESULT_BYTES, dtype=torch.uint8, device=Od.device)
    ctx.single_async(Od, out, prec=prec)
    torch.cuda.synchronize()
    ctx.set_timing(True)
    ms = []
    for _ in range(reps):
        ctx.single_async(Od, out, prec=prec)
        ms.append(ctx.walk_time_ms())
    ctx.set_timing(False)
    return ms, tor.TorResult.from_bytes(out.cpu().numpy().tobytes())


def k50_projection(ctx, rng_seed=3, windows=2):
    """Config 3's k = 50 Torontonian (M = 100, r ~ U[0.8, 1.4], eta = 0.3, seed 3): the bound
    pass routes it, random windows of its chunks are walked at that tier (one warm-up), and the
    full 2^50-subset runtime is projected from the mean rate."""
    import math
    import torch
    from paper_2009_01177_gb300 import gbs_inputs as gi
    st = gi.lossy_gbs_state(100, 0.8, 1.4, 0.3, 3)
    pat = gi.random_pattern(100, 50, 1003)
    k = 50
    Od = torch.from_numpy(gi.select(st.O, pat[:k])).cuda()
    bd = ctx.bounds([Od], tol=1e-10)[0]
    tier = TIER_NAME[int(bd["tier"])]
    r1 = {"fp64": 16, "dd": 13, "fx128": 13, "fx256": 17}[tier]
    window = 1 << 17
    d = k - r1
    rng = np.random.default_rng(rng_seed)
    ms = []
    for w in range(windows + 1):
        c0 = int(rng.integers(0, (1 << d) // window)) * window
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.chunks(Od, d, c0, c0 + window, prec=tier)
        e1.record()
        torch.cuda.synchronize()
        if w:
            ms.append(e0.elapsed_time(e1))
    rate = window * (1 << r1) / (float(np.mean(ms)) * 1e-3)
    return {"workload": "k=50 pattern (100x100 O_S) of the M=100 state r~U[0.8,1.4], eta=0.3, seed 3",
            "routed_tier": tier, "bits_needed": float(bd["bits_needed"]),
            "log2_tmax": float(bd["log_tmax"]) / math.log(2), "chunk_bits": d, "window_chunks": window,
            "windows_ms": [round(x, 1) for x in ms], "subset_dets_per_s": rate,
            "projected_full_s": 2.0 ** k / rate,
            "paper_context_s": {"128-bit, 39,286 TaihuLight nodes": 73773, "256-bit, same": 170891}}


def run_single(args):
    """One Torontonian per step, routed by the bound pass to the tier that resolves it and
    checked against tol; on N > 1 ranks the chunks of that one Torontonian are split."""
    import math
    import torch
    rank, world, local = env_rank()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2009_01177_gb300 import tor
    k, tol = args.k, args.tol
    st, pat, O = workload(k, 0)
    ctx = tor.Context(local)
    Od = torch.from_numpy(O).to(dev)
    bd = ctx.bounds([Od], tol=tol)[0]
    routed = TIER_NAME[int(bd["tier"])]
    tier = routed if args.prec == "auto" else args.prec
    route = {"tol": tol, "requested": args.prec, "routed_tier": routed,
             "bits_needed": float(bd["bits_needed"]), "log2_tmax": float(bd["log_tmax"]) / math.log(2),
             "log2_kappa_est": float(bd["log_kappa_est"]) / math.log(2)}
    if args.chunk_bits is None:
        # the project's autotuner picks the chunk depth and blocks per SM for this k and tier
        tuned_d, tuned_bps = ctx.autotune(k, tier)
        launch_how = "autotuned"
    else:
        tuned_d, tuned_bps = args.chunk_bits, args.blocks_per_sm
        ctx.set_chunk_bits(tuned_d)
        ctx.set_launch(128, tuned_bps)
        launch_how = "given"
    if world > 1:
        # every rank must cut the subsets into the same chunks: rank 0's depth for all
        import torch.distributed as dist
        dt = torch.tensor([tuned_d], dtype=torch.int64, device=dev)
        dist.broadcast(dt, 0)
        return run_sharded(args, ctx, Od, k, tier, int(dt.item()), route, rank, world, dev)

    peak_dfma, clk = ctx.fp64_peak()
    peak_mad = ctx.int_peak()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        ctx.single(Od, prec=args.prec, tol=tol)
    torch.cuda.synchronize()

    ctx.set_timing(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    walk_ms, results = [], []
    with ClockSampler(local) as clocks:
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record()
            results.append(ctx.single(Od, prec=args.prec, tol=tol))   # bound pass, walk, result to host
            ev[i][1].record()
            walk_ms.append(ctx.walk_time_ms())
        torch.cuda.synchronize()
    ctx.set_timing(False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(step_ms) / 1e3
    res = results[-1]

    # end to end: pinned host input -> device, the same call, the result on the host; wall clock
    O_pin = torch.from_numpy(O).pin_memory()
    Od2 = torch.empty_like(Od)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        Od2.copy_(O_pin, non_blocking=True)
        r_e2e = ctx.single(Od2, prec=args.prec, tol=tol)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0

    # the FP64 walk on the same instance: kernel quality only, it does not resolve this kappa
    fp64 = None
    if not args.no_fp64 and tier != "fp64":
        if args.chunk_bits is None:
            ctx.autotune(k, "fp64")
        ms64, r64 = _timed_walks(ctx, Od, "fp64", 3)
        w64 = float(np.mean(ms64))
        t64 = FLOPS_PER_SUBSET * 2 ** k / (w64 * 1e-3) / 1e12
        fp64 = {"kernel": "k_dfs<TierF64>", "subset_dets_per_s": 2 ** k / (w64 * 1e-3), "kernel_ms": w64,
                "tflops": t64, "frac_of_fp64_peak": t64 / PEAK_TFLOPS,
                "measured_dfma_tflops": 2 * peak_dfma / 1e12, "flops_per_subset": FLOPS_PER_SUBSET,
                "err_est_over_tor": r64.err_est / abs(r64.value) if r64.value else None,
                "resolved": bool(r64.err_est <= tol * abs(r64.value)),
                "traffic": recorded_traffic("k_dfs_fp64", k),
                "note": "FP64 tier timed on the same instance; its error bound exceeds |Tor| at this "
                        "kappa, so it is a kernel-quality figure, not a Torontonian"}

    k50 = None if args.no_k50 else k50_projection(ctx)

    units = float(2 ** k) * args.steps
    value = units / total_s
    walk_avg = float(np.mean(walk_ms))
    resolved = bool(res.status == 0 and res.err_est <= tol * abs(res.value))
    kernel = "k_dfs_fx9" if res.tier == 4 else "k_dfs<%s>" % TIER_NAME[res.tier]
    if res.tier == 4:
        macs = fx256_macs_per_subset(k)
        achieved = macs * 2 ** k / (walk_avg * 1e-3) / 1e12
        traffic = recorded_traffic("k_dfs_fx9", k)
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak_mad / 1e12, "unit": "T int32-MAC/s",
                    "frac": achieved / (peak_mad / 1e12), "traffic": traffic, "kernel": kernel,
                    "kernel_ms": walk_avg,
                    "peak_source": "measured: independent mad.wide.s32 chains on all SMs (tor_int_peak), "
                                   "the limb product of the 256-bit-class arithmetic",
                    "macs_per_subset": macs,
                    "derivation": "per subset: 2x2 det 2 + rsqrt step 2 + term 1 products, 0.5 "
                                  "coefficient sets x 4, 2 pivot rows x 4, 7 Schur entries x 2 = 29 "
                                  "products of 60 limb MACs, plus the rsqrt step's 18-MAC short "
                                  "product (walk over all 2^k subsets); the seed runs on the FP64 pipe",
                    "dram": dram_rate(traffic, walk_avg)}
    else:
        achieved = FLOPS_PER_SUBSET * 2 ** k / (walk_avg * 1e-3) / 1e12
        traffic = recorded_traffic("k_dfs_fp64", k) if res.tier == 1 else None
        roofline = {"bound": "alu", "achieved": achieved, "peak": PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / PEAK_TFLOPS, "traffic": traffic, "kernel": kernel,
                    "kernel_ms": walk_avg, "peak_source": "derived: 2 DFMA/clk/SM x 152 SMs x 2.07 GHz x 2",
                    "flops_per_subset": FLOPS_PER_SUBSET}
    cpu = None
    if not args.no_cpu_baseline:
        n, el, nch = cpu_oracle_sample(O, k, budget_s=args.cpu_budget)
        cpu = {"value": n / el, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{nch} random 256-subset chunks (masks [c 2^8, (c+1) 2^8)) of the same "
                         f"k={k} matrix, {el:.1f} s; 256-bit fixed point, OpenMP over masks"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_OF[TIER_NAME[res.tier]], "data": "synthetic",
        "config": config(k, {"tier": TIER_NAME[res.tier], "route": route, "chunk_bits": tuned_d,
                             "blocks_per_sm": tuned_bps, "launch": launch_how}),
        "e2e": {"value": units / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(O.nbytes),
                "d2h_bytes_per_step": tor.RESULT_BYTES},
        "gpu_launches": 4 * args.steps,
        "roofline": roofline,
        "fp64_walk": fp64,
        "k50_projection": k50,
        "paper_equivalent": {"tflops": paper_flops(k) / (walk_avg * 1e-3) / 1e12, "flops_per_launch": paper_flops(k),
                             "note": "the paper's FLOP count of Eq. tflops (a fresh complex solve per "
                                     "subset) over the walk time"},
        "cpu_baseline": cpu,
        "clocks": clocks.summary(),
        "result": {"tor": res.value, "hi": res.hi, "lo": res.lo, "sum_abs": res.sum_abs,
                   "err_est": res.err_est, "err_est_over_tor": res.err_est / abs(res.value) if res.value else None,
                   "kappa": res.kappa, "tier": TIER_NAME[res.tier], "resolved": resolved,
                   "steps_identical": len({(r.hi, r.lo) for r in results}) == 1,
                   "e2e_equal": (r_e2e.hi, r_e2e.lo) == (res.hi, res.lo)},
    }
    print(json.dumps(line), flush=True)
    ctx.close()
    if not resolved:
        sys.stderr.write(f"error bound {res.err_est:.3e} exceeds tol * |Tor| = {tol * abs(res.value):.3e}\n")
        sys.exit(3)


def run_sharded(args, ctx, Od, k, tier, d, route, rank, world, dev):
    """N > 1: the 2^d chunks of the one Torontonian split over the ranks (Algorithm 1's rank
    partition), each rank's exact partial sum all-gathered and added (the only exchange)."""
    import torch
    import torch.distributed as dist
    from paper_2009_01177_gb300 import shard, tor

    def step():
        r, _ = shard.tor_sharded(ctx, Od, d, tier)
        return r

    for _ in range(args.warmup):
        step()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(int(os.environ.get("LOCAL_RANK", 0))) as clocks:
        dist.barrier()
        torch.cuda.synchronize()
        for i in range(args.steps):
            ev[i][0].record()
            res = step()
            ev[i][1].record()
        dist.barrier()
        torch.cuda.synchronize()
    total_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    total_s, = max_over_ranks([total_s], world, dev)
    resolved = bool(res.status == 0 and res.err_est <= args.tol * abs(res.value))
    if rank == 0:
        units = float(2 ** k) * args.steps
        line = {"metric": METRIC, "value": units / total_s, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": DTYPE_OF[tier], "data": "synthetic",
                "config": config(k, {"tier": tier, "route": route, "chunk_bits": d,
                                     "parallelism": f"chunk ranges over {world} ranks, exact all-gather",
                                     "l2": "not flushed (the sharded step's inputs are one 2k x 2k matrix)"}),
                "gpu_launches": 3 * args.steps,
                "clocks": clocks.summary(),
                "result": {"tor": res.value, "err_est": res.err_est, "tier": tier, "resolved": resolved}}
        print(json.dumps(line), flush=True)
    ctx.close()
    dist.destroy_process_group()
    if not resolved:
        sys.exit(3)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--k", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--mode", default="single", choices=["single", "batch", "mh", "adaptive", "table", "levels"])
    ap.add_argument("--table-m", type=int, default=26, help="table mode: modes M (2^M patterns)")
    ap.add_argument("--prec", default="auto", choices=["auto", "fp64", "dd", "fx128", "fx256"],
                    help="single mode: AUTO (the bound pass routes to the tier that meets --tol, escalating "
                         "on the a-posteriori bound) or an explicit tier")
    ap.add_argument("--tol", type=float, default=1e-10, help="relative tolerance every result must meet")
    ap.add_argument("--no-fp64", action="store_true", help="single mode: skip the secondary FP64 walk timing")
    ap.add_argument("--no-k50", action="store_true", help="single mode: skip the k = 50 runtime projection")
    ap.add_argument("--full-k40", action="store_true", help="adaptive mode: also run the whole k = 40 Torontonian")
    ap.add_argument("--n", type=int, default=4096, help="patterns (batch) or chains (mh)")
    ap.add_argument("--patterns", default="marginals", choices=["marginals", "chainrule"],
                    help="batch mode: independent clicks with the exact marginals, or exact chain-rule "
                         "samples (about 2e12 subset determinants per 2048 samples)")
    ap.add_argument("--mh-tol", type=float, default=1e-8, help="mh mode: tolerance of every exact Torontonian")
    ap.add_argument("--chunk-bits", type=int, default=None,
                    help="single mode: chunk depth d instead of the autotuner's choice")
    ap.add_argument("--blocks-per-sm", type=int, default=4, help="with --chunk-bits: resident blocks per SM")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    if args.impl == "reference":
        run_reference(args)
        return
    if args.mode == "batch":
        run_batch(args)
        return
    if args.mode == "mh":
        run_mh(args)
        return
    if args.mode == "adaptive":
        run_adaptive(args)
        return
    if args.mode == "table":
        run_table(args)
        return
    if args.mode == "levels":
        run_levels(args)
        return

    run_single(args)


if __name__ == "__main__":
    main()
