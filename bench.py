#!/usr/bin/env python
"""Benchmark: AD-PRD operator applies/s on the Mg II h&k-like workload
(70 heights x 64 directions x 200 wavelengths, N = 3.58e6 unknowns, FP32),
plus one preconditioned GMRES solve, as one JSON line on stdout.

A step is one operator apply y = (Id - Lambda Sigma) x (all stages S1-S8 of
the hot path) on inputs resident in HBM.  N > 1 GPUs (torchrun, one rank per
GPU) run independent instances (weak scaling, no data-path collective).

--impl reference times the FP64 CPU oracle on bounded samples of the same
workload (Sigma rows at a few (height, direction) pairs plus formal-solution
rays), scaled to one full apply.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# the CPU oracle legs report one core: keep numpy's BLAS single-threaded
for _v in ("OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np   # noqa: E402

METRIC = "AD-PRD operator applies/s, GMRES solve s at 1e-5 rel err; % of roofline"
UNIT = "applies/s"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return PEAKS_FALLBACK, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([s.strip() for s in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) > 8 for i in range(4)
                          if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def oracle_problem(cfg):
    """The oracle's set-up for the workload (atom, K, DELO tables); not timed."""
    from oracle.problem import Problem
    return Problem(cfg, normalise=False)


def oracle_sample(P, n_dirs_in=4, n_rays=64, seed=5):
    """Time the oracle on a bounded sample; return (seconds per full apply, description).
    Its tile caches are emptied first, so every sample computes its tiles."""
    P._tiles.clear()
    P._r3.clear()
    x = np.random.default_rng(seed).uniform(0.1, 1.0, P.shape())
    iz, o = P.nz // 2, P.nO - 3
    t0 = time.perf_counter()
    sb = np.zeros((P.nN, 4))
    for op in range(n_dirs_in):
        blk = P.block(iz, o, op).reshape(P.nN * 4, P.nN * 4)
        sb += (blk @ (P.interp_in(iz, op) @ x[iz, op]).ravel()).reshape(P.nN, 4)
    eps = P.interp_back(iz, o) @ sb
    t_sig = (time.perf_counter() - t0) * P.nO / n_dirs_in          # one (z, Omega) row, all Omega'
    t0 = time.perf_counter()
    for r in range(n_rays):
        P.lambda_ray(x, r % P.nO, (7 * r) % P.nN)
    t_lam = (time.perf_counter() - t0) / n_rays * P.nO * P.nN
    per_apply = t_sig * P.nz * P.nO + t_lam
    desc = (f"oracle Sigma row at 1 (height, direction) with {n_dirs_in} of {P.nO} incident directions "
            f"(scaled x{P.nO // n_dirs_in}), times {P.nz}x{P.nO} rows, plus Lambda on {n_rays} of "
            f"{P.nO * P.nN} rays (scaled); tile setup of the sampled rows included")
    return per_apply, desc, float(eps[0, 0])


def max_over_ranks(ms, dist, device):
    """The job's time: the largest per-rank time over the ranks (any backend)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, ms):
    """Whole-job applies/s: every rank applies its own instance once per step."""
    return world * 1e3 / ms


def run_reference(args, cfg, workload):
    threads = 1
    per = []
    desc = ""
    P = oracle_problem(cfg)
    for step in range(args.warmup + args.steps):
        t, desc, _ = oracle_sample(P, n_dirs_in=1 if step < args.warmup else 2, seed=step)
        if step >= args.warmup:
            per.append(t)
    value = 1.0 / statistics.median(per)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--solve-tol", type=float, default=1e-10,
                    help="GMRES tol; 1e-10 is the largest meeting 1e-5 on emergent I in the Mg II parity case")
    ap.add_argument("--workload", default="mgii", choices=["mgii", "mgii_small"],
                    help="mgii_small (8 heights) is only for ncu captures of single kernels")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    from paper_2505_20968_gb300 import inputs
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cfg = inputs.mgii(seed=2 + rank) if args.workload == "mgii" else inputs.mgii(n_z=8, seed=2 + rank)
    nz, nnu = len(cfg["atm"]["z_km"]), len(cfg["quad"]["grid"])
    nmu, nchi = cfg["quad"]["n_mu_half"], cfg["quad"]["n_chi"]
    workload = {"workload": f"mgii_hk_like: two-term Mg II h&k, {nz} heights, {nnu} wavelengths, "
                            f"{nmu}+{nmu} GL mu x {nchi} chi ({2 * nmu * nchi} directions), B<=100 G, |v|<=5 km/s, "
                            f"N={4 * nz * nnu * 2 * nmu * nchi:,}",
                "precision": "fp32 tiles/vectors, fp64 reductions", "parallelism": f"{world} independent instances",
                "l2": "inputs larger than L2 (R_II tiles ~40 GB streamed per apply)"}
    if args.impl == "reference":
        if rank == 0:
            run_reference(args, cfg, workload)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2505_20968_gb300.binding import PRD

    t0 = time.time()
    P = PRD(cfg, device=local)
    torch.cuda.synchronize()
    setup_s = time.time() - t0
    g = torch.Generator(device="cuda").manual_seed(1234 + rank)
    x = torch.rand(P.shape, device="cuda", dtype=P.dtype, generator=g)
    x[..., 1:] *= 0.05
    y = P.empty()
    for _ in range(args.warmup):
        P.apply_operator(x, y)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        P.apply_operator(x, y)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, "cuda")
    value = job_value(world, ms)

    # end to end through the public API with host buffers (pinned), copies timed
    xh = x.cpu().pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    xd = torch.empty_like(x)
    for _ in range(2):
        xd.copy_(xh, non_blocking=True)
        P.apply_operator(xd, y)
        yh.copy_(y, non_blocking=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        xd.copy_(xh, non_blocking=True)
        P.apply_operator(xd, y)
        yh.copy_(y, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, "cuda")
    nbytes = x.numel() * x.element_size()

    # per-stage durations (CUDA events on the library stream) for the roofline
    P.set_profiling(True)
    for _ in range(3):
        P.apply_operator(x, y)
    st = P.stage_times()
    P.set_profiling(False)
    r2_ms = st["S3_R2_contraction"][0] / max(st["S3_R2_contraction"][1], 1)
    flops, tile_bytes = P.contraction_work()
    peaks, src = _peaks()
    # The contraction runs 3 TF32 products per FP32-accurate product (hi*hi + hi*lo +
    # lo*hi); its tensor time at peak exceeds the HBM time of streaming the tiles, so
    # the tensor pipe at the TF32 rate bounds it.  TF32 peak = measured bf16 peak x
    # the nominal dense TF32 / bf16 ratio (1.1 / 2.25 PFLOP/s).
    tf32_peak = peaks["bf16_tflops"] * (1.1 / 2.25)
    achieved_tf = 3.0 * flops / (r2_ms * 1e-3) / 1e12
    achieved_gbs = tile_bytes / (r2_ms * 1e-3) / 1e9
    traffic = None
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            tr = json.load(f)
        if tr.get("kernel") == "r2_tc_kernel" and tr.get("workload") == "mgii" and tr.get("layout") == "bulk-v3":
            traffic = tr.get("dram_bytes_per_launch")
    except (OSError, ValueError):
        pass
    roofline = {"bound": "tensor", "kernel": "r2_tc_kernel (S3+S4 R_II contraction, tcgen05 3xTF32)",
                "achieved": achieved_tf, "peak": tf32_peak, "unit": "TFLOP/s", "frac": achieved_tf / tf32_peak,
                "peak_source": src + " bf16 x nominal tf32/bf16 ratio", "traffic": traffic,
                "algorithmic_flops_per_launch": 3.0 * flops, "algorithmic_bytes_per_launch": tile_bytes,
                "hbm": {"achieved": achieved_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": achieved_gbs / peaks["hbm_gbs"]},
                "launch_ms": r2_ms, "stage_ms": {k: v[0] / max(v[1], 1) for k, v in st.items()}}

    solve = None
    if not args.no_solve:
        torch.cuda.synchronize()
        t0 = time.time()
        sol, info = P.solve(tol=args.solve_tol, max_iter=600, restart=60, check=False)
        torch.cuda.synchronize()
        solve = {"seconds": time.time() - t0, "tol": args.solve_tol, "applies": info["iters"],
                 "true_rel_res": info["true_rel_res"], "rc": info["rc"], "setup_seconds": setup_s}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        per, desc, _ = oracle_sample(oracle_problem(cfg))
        cpu = {"value": 1.0 / per, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload,
                "clocks": clk,
                "e2e": {"value": job_value(world, ms_e2e), "unit": UNIT, "h2d_bytes_per_step": nbytes,
                        "d2h_bytes_per_step": nbytes},
                "gpu_launches": 8 * args.steps, "roofline": roofline, "cpu_baseline": cpu, "solve": solve}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
