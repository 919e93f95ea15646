#!/usr/bin/env python
"""Benchmark: subset determinants per second of the Torontonian on one click pattern.

Workload: the Torontonian of a k = 32 click pattern (64 x 64 FP64 matrix,
2^32 subsets) of a synthetic M = 100 mode lossy GBS state (r ~ U[0.6, 1.2],
Haar U, eta = 0.3, seed 2), FP64 tier.  One step = one full Torontonian:
prep (I - O, basis) + chunk roots + depth-first walk + exact reduction.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line on rank 0.  Under torchrun (N > 1) each rank evaluates
the Torontonian of its own click pattern of the same state (independent
problems, no data-path collective: weak scaling).

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


def workload(k, rank):
    from paper_2009_01177_gb300 import gbs_inputs as gi
    st, pat, O = gi.workload_m100(k, seed=2, pattern_seed=None if rank == 0 else 2000 + rank)
    return st, pat, O


def config(k, extra=None):
    c = {"workload": f"single Torontonian k={k} ({2 * k}x{2 * k} FP64 O_S) of a synthetic M=100 lossy "
                     f"GBS state (r~U[0.6,1.2], Haar U, eta=0.3, seed 2)",
         "k": k, "subsets_per_step": 2 ** k, "tier": "fp64",
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
            "data": "synthetic", "config": config(k, {"tier": "oracle (256-bit fixed point, CPU)"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--k", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    rank, world, local = env_rank()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2009_01177_gb300 import tor
    k = args.k
    st, pat, O = workload(k, rank)
    ctx = tor.Context(local)
    peak_dfma, clk = ctx.fp64_peak()
    Od = torch.from_numpy(O).to(dev)
    out = torch.empty(tor.RESULT_BYTES, dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    for _ in range(args.warmup):
        ctx.single_async(Od, out, prec="fp64")
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    ctx.set_timing(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    walk_ms = []
    with ClockSampler(local) as clocks:
        barrier()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record()
            ctx.single_async(Od, out, prec="fp64")
            ev[i][1].record()
            walk_ms.append(ctx.walk_time_ms())
        barrier()
    ctx.set_timing(False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(step_ms) / 1e3
    res = tor.TorResult.from_bytes(out.cpu().numpy().tobytes())

    # end to end: pinned host input -> device, call, host result; wall clock
    O_pin = torch.from_numpy(O).pin_memory()
    Od2 = torch.empty_like(Od)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        Od2.copy_(O_pin, non_blocking=True)
        r_e2e = ctx.single(Od2, prec="fp64")
    barrier()
    e2e_s = time.perf_counter() - t0

    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([total_s, e2e_s], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s, e2e_s = float(t[0]), float(t[1])

    if rank == 0:
        units = float(2 ** k) * args.steps * world
        value = units / total_s
        walk_avg = sum(walk_ms) / len(walk_ms)
        achieved = FLOPS_PER_SUBSET * 2 ** k / (walk_avg * 1e-3) / 1e12
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            n, el, nch = cpu_oracle_sample(O, k, budget_s=args.cpu_budget)
            cpu = {"value": n / el, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"{nch} random 256-subset chunks (masks [c 2^8, (c+1) 2^8)) of the same "
                             f"k={k} matrix, {el:.1f} s; 256-bit fixed point, OpenMP over masks"}
        traffic = None
        prof = os.path.join(ROOT, "profiles", "traffic.json")
        if os.path.exists(prof):
            try:
                traffic = json.load(open(prof)).get(f"k_dfs_fp64_k{k}")
            except (OSError, ValueError):
                traffic = None
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config(k, {"fp64_peak_frac": achieved / PEAK_TFLOPS}),
            "e2e": {"value": float(2 ** k) * args.steps * world / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": int(O.nbytes), "d2h_bytes_per_step": tor.RESULT_BYTES},
            "gpu_launches": 3 * args.steps,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / PEAK_TFLOPS, "traffic": traffic,
                         "kernel": "k_dfs<TierF64>", "kernel_ms": walk_avg,
                         "peak_source": "derived: 2 DFMA/clk/SM x 152 SMs x 2.07 GHz x 2 flops",
                         "measured_dfma_tflops": 2 * peak_dfma / 1e12,
                         "flops_per_subset": FLOPS_PER_SUBSET},
            "cpu_baseline": cpu,
            "clocks": clocks.summary(),
            "result": {"tor": res.value, "sum_abs": res.sum_abs, "err_est": res.err_est,
                       "kappa": res.kappa, "e2e_equal": (r_e2e.hi, r_e2e.lo) == (res.hi, res.lo)},
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
