"""Benchmark: exprb53 steps/s on the level-7 icosahedral shallow-water grid.

One step = one exprb53 step (Sec. 3.3, Eq. eq3.13; three phipm_simul_iom2
calls, Sec. 4.4) of the FP64 path on a seeded balanced state (163842 cells,
n = 655368, dt = 3600 s, Tol = 1e-8 relative), every stage on the GPU.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line.  value = whole-job steps/s (N independent replicas under
torchrun: the path has no data-parallel exchange); e2e = the same metric
through the public API from pinned host memory and back; roofline = the
persistent phipm_simul_iom2 kernel (FP64-ALU bound) from CUDA events recorded
by the library on the launching stream; cpu_baseline = the FP64 oracle timed
on one host core on a bounded sample (one step).  --impl reference times the
oracle itself as the reference arm.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

LEVEL, SCHEME, DT, SEED, AMP, TOL = 7, "exprb53", 3600.0, 2, 400.0, 1e-8
METRIC = "exprb53 steps/s (level-7 SWE)"
UNIT = "steps/s"
# FP64 peak: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2.07 GHz (the unit count a
# dependent-chain-free FMA probe reproduces: 1.196 TFLOP/s at ~1.97 GHz).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
WORKLOAD = ("exprb53 step, level-7 icosahedral geodesic grid (163842 cells, n=655368), "
            "dt=3600 s, FP64, IOM2 Tol=1e-8 relative, m_max=64, seeded balanced state "
            "(seed 2, 400 m)")


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def _traffic():
    """DRAM bytes per phi launch from the committed ncu summary (None if absent or stale)."""
    p = os.path.join(ROOT, "profiles", "phi_kernel_traffic.json")
    try:
        d = json.load(open(p))
        return d.get("dram_bytes_per_launch")
    except Exception:
        return None


def _config():
    return {"workload": WORKLOAD, "level": LEVEL, "scheme": SCHEME, "dt": DT, "precision": "fp64",
            "tol": TOL, "l2": "L2 (129 MB) flushed with a 256 MB write between timed steps; "
            "the Krylov basis (~340 MB) exceeds L2", "parallelism": "replicas"}


# ---------------------------------------------------------------------------
# oracle sample (CPU baseline / reference arm)
# ---------------------------------------------------------------------------
def oracle_steps(nsteps: int, warmup: int) -> dict:
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle.phipm import PhiOpts
    from oracle.schemes import KrylovPhi, step
    from oracle.swe import make_swe
    from paper_1805_02144_gb300.inputs import balanced_state
    s = make_swe(LEVEL)
    u = balanced_state(s.grid.x, SEED, AMP)
    kp = KrylovPhi(s, PhiOpts(tol=TOL))
    for _ in range(warmup):
        u = step(SCHEME, s, u, DT, kp)
    times = []
    for _ in range(nsteps):
        t0 = time.perf_counter()
        u = step(SCHEME, s, u, DT, kp)
        times.append(time.perf_counter() - t0)
    return {"times": times}


def run_oracle_subprocess(nsteps: int, warmup: int) -> dict:
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = (f"import json,sys; sys.path.insert(0, {ROOT!r}); import bench; "
            f"print(json.dumps(bench.oracle_steps({nsteps}, {warmup})))")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=1800)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def reference_arm(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    res = run_oracle_subprocess(args.steps, min(args.warmup, 1))
    total = sum(res["times"])
    value = args.steps / total
    sample = (f"{args.steps} oracle {SCHEME} steps of the level-7 workload after "
              f"{min(args.warmup, 1)} untimed step (numpy/scipy FP64, one thread)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": _config(),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for nme, v in zip(names, parts[2:6]):
                if v.lower().startswith("active"):
                    reasons.add(nme)
        if not sm:
            return None
        loaded = [x for x in sm if x > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def gpu_arm(args) -> None:
    import numpy as np
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1805_02144_gb300 import build
    build.build()
    from paper_1805_02144_gb300.api import (Grid, SchemeState, exprb_step, swe_profile_enable,
                                            swe_profile_read)
    from paper_1805_02144_gb300.inputs import balanced_state

    G = Grid(LEVEL)
    u0 = torch.from_numpy(balanced_state(G.cell_centres(), SEED, AMP)).cuda()
    st = SchemeState(G)
    opts = {"tol": TOL}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    bufs = [u0.clone(), torch.empty_like(u0)]

    sampler = ClockSampler(local)
    for k in range(args.warmup):
        exprb_step(G, SCHEME, DT, bufs[k % 2], out=bufs[(k + 1) % 2], state=st, opts=opts)
    cur = args.warmup % 2
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    swe_profile_enable(G, True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        exprb_step(G, SCHEME, DT, bufs[cur], out=bufs[1 - cur], state=st, opts=opts)
        ev[k][1].record(stream)
        cur = 1 - cur
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    prof = swe_profile_read(G)
    swe_profile_enable(G, False)
    t_ms = sum(a.elapsed_time(b) for a, b in ev)
    if dist:
        t = torch.tensor([t_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_ms = float(t.item())
    value = world * args.steps / (t_ms / 1e3)

    # end to end through the public API: pinned host state in, host state out
    n = G.n
    h_in = torch.empty(n, dtype=torch.float64, pin_memory=True)
    h_in.copy_(bufs[cur].cpu())
    h_out = torch.empty(n, dtype=torch.float64, pin_memory=True)
    d_in, d_out = torch.empty_like(u0), torch.empty_like(u0)
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    for k in range(args.steps):
        flush.fill_(float(k))
        ev2[k][0].record(stream)
        d_in.copy_(h_in, non_blocking=True)
        exprb_step(G, SCHEME, DT, d_in, out=d_out, state=st, opts=opts)
        h_out.copy_(d_out, non_blocking=True)
        ev2[k][1].record(stream)
        ev2[k][1].synchronize()
        h_in, h_out = h_out, h_in
    torch.cuda.synchronize()
    e_ms = sum(a.elapsed_time(b) for a, b in ev2)
    if dist:
        t = torch.tensor([e_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e_ms = float(t.item())
    e2e = world * args.steps / (e_ms / 1e3)
    finite = bool(torch.isfinite(bufs[cur]).all().item())

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    phi_launch_ms = prof["phi_ms"] / max(prof["phi_launches"], 1)
    achieved = prof["phi_flop"] / (prof["phi_ms"] / 1e3) / 1e12
    peaks = _peaks()
    hbm = peaks.get("hbm_gbs")
    traffic = _traffic()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(),
        "roofline": {
            "kernel": "phi_kernel (persistent phipm_simul_iom2 launch)",
            "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS,
            "traffic": traffic,
            "peak_source": "FP64 unit count x max clock (152 SMs x 4 flop/clk x 2.07 GHz)",
            "launch_ms": phi_launch_ms, "launches": prof["phi_launches"],
            "share_of_step": prof["phi_ms"] / t_ms,
            "algorithmic_flop_per_launch": prof["phi_flop"] / max(prof["phi_launches"], 1),
            "hbm_gbs_algorithmic": prof["phi_bytes"] / (prof["phi_ms"] / 1e3) / 1e9,
            "hbm_frac_of_measured": (prof["phi_bytes"] / (prof["phi_ms"] / 1e3) / 1e9 / hbm) if hbm else None,
            "iom2_iterations_per_step": prof["iom2_iterations"] / args.steps,
            "phase_ms_per_step": {k: v / args.steps for k, v in prof["phase_ms"].items()},
        },
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n},
        "gpu_launches": prof["kernel_launches"],
        "clocks": clocks,
        "finite": finite,
    }
    if world == 1 and not args.no_cpu_baseline:
        try:
            res = run_oracle_subprocess(1, 0)
            cb = 1.0 / res["times"][0]
            line["cpu_baseline"] = {"value": cb, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": "one oracle exprb53 step of the same level-7 "
                                              "workload from the initial state (numpy/scipy FP64, "
                                              "one thread)"}
        except Exception as e:  # report, do not hide
            line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": f"failed: {e!s:.200}"}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
