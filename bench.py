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

import numpy as np
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
    """DRAM bytes per phi launch from the committed ncu summary; None if absent
    or if the kernel's source files changed since the counters were taken."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "phi_kernel_traffic.json")
    try:
        d = json.load(open(p))
        h = hashlib.sha256()
        for f in d["source_files"]:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        if h.hexdigest() != d["source_sha256"]:
            return None
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


def run_oracle_subprocess(nsteps: int, warmup: int, threads: int = 1) -> dict:
    t = str(threads)
    env = dict(os.environ, OMP_NUM_THREADS=t, OPENBLAS_NUM_THREADS=t, MKL_NUM_THREADS=t)
    code = (f"import json,sys; sys.path.insert(0, {ROOT!r}); import bench; "
            f"print(json.dumps(bench.oracle_steps({nsteps}, {warmup})))")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=1800)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_replica_step(ready_dir: str, rank: int) -> None:
    """One oracle step of the workload, started when every replica is ready
    (used by oracle_replicas): prints its wall-clock start and end."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle.phipm import PhiOpts
    from oracle.schemes import KrylovPhi, step
    from oracle.swe import make_swe
    from paper_1805_02144_gb300.inputs import balanced_state
    s = make_swe(LEVEL)
    u = balanced_state(s.grid.x, SEED, AMP)
    kp = KrylovPhi(s, PhiOpts(tol=TOL))
    open(os.path.join(ready_dir, f"ready{rank}"), "w").close()
    go = os.path.join(ready_dir, "go")
    t_wait = time.time()
    while not os.path.exists(go):
        if time.time() - t_wait > 600:
            raise RuntimeError("replica start timed out")
        time.sleep(0.01)
    t0 = time.time()
    step(SCHEME, s, u, DT, kp)
    print(json.dumps({"t0": t0, "t1": time.time()}), flush=True)


def oracle_replicas(nproc: int) -> dict:
    """The oracle on every host core: nproc independent processes (one thread
    each) run one step of the same workload at the same time; the combined
    rate is nproc steps over the span from the first start to the last end."""
    import tempfile
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    with tempfile.TemporaryDirectory() as d:
        procs = []
        for r in range(nproc):
            code = (f"import sys; sys.path.insert(0, {ROOT!r}); import bench; "
                    f"bench.oracle_replica_step({d!r}, {r})")
            procs.append(subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE,
                                          stderr=subprocess.PIPE, text=True, env=env))
        t_wait = time.time()
        while sum(os.path.exists(os.path.join(d, f"ready{r}")) for r in range(nproc)) < nproc:
            if time.time() - t_wait > 600 or any(p.poll() not in (None, 0) for p in procs):
                for p in procs:
                    p.kill()
                raise RuntimeError("oracle replicas did not start")
            time.sleep(0.05)
        open(os.path.join(d, "go"), "w").close()
        spans = []
        for p in procs:
            out, err = p.communicate(timeout=1800)
            if p.returncode != 0:
                raise RuntimeError(err[-1000:])
            spans.append(json.loads(out.strip().splitlines()[-1]))
    t0 = min(x["t0"] for x in spans)
    t1 = max(x["t1"] for x in spans)
    return {"value": nproc / (t1 - t0), "span_s": t1 - t0,
            "step_s": [x["t1"] - x["t0"] for x in spans]}


def reference_arm(args) -> None:
    from paper_1805_02144_gb300.ranks import from_env
    if not from_env().lead:  # the oracle runs once, on rank 0
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
def timed_steps(G, u0, scheme, dt, nsteps, opts, flush, state=None, profile=False):
    """nsteps steps from u0, one CUDA event pair per step on the current stream
    (L2 flushed between steps outside the events).  Returns (per-step ms list,
    final state, profile dict or None)."""
    import torch
    from paper_1805_02144_gb300.api import (SchemeState, exprb_step, swe_profile_enable,
                                            swe_profile_read)
    st = state if state is not None else SchemeState(G)
    stream = torch.cuda.current_stream()
    bufs = [u0.clone(), torch.empty_like(u0)]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(nsteps)]
    if profile:
        swe_profile_enable(G, True)
    torch.cuda.synchronize()
    cur = 0
    for k in range(nsteps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        exprb_step(G, scheme, dt, bufs[cur], out=bufs[1 - cur], state=st, opts=opts)
        ev[k][1].record(stream)
        cur = 1 - cur
    torch.cuda.synchronize()
    prof = None
    if profile:
        prof = swe_profile_read(G)
        swe_profile_enable(G, False)
    return [a.elapsed_time(b) for a, b in ev], bufs[cur], prof


def precision_block(flush) -> dict:
    """Mixed precision vs FP64 on the level-8 exprb53 12 h run (same state),
    and the same comparison on the level-9 grid."""
    out = precision_run(flush, 8)
    try:
        lv9 = precision_run(flush, 9)
        out["level9"] = {k: lv9[k] for k in ("workload", "mixed", "fp64", "speedup_mixed_over_fp64",
                                             "rel_l2_mixed_vs_fp64", "rel_l2_mixed_vs_fp64_same_tol",
                                             "rel_l2_fp64_tol_1e-6_vs_1e-8")}
    except Exception as e:  # recorded, never fatal to the bench line
        out["level9"] = {"error": f"{e!s:.300}"}
    return out


def precision_run(flush, level: int) -> dict:
    import torch
    from paper_1805_02144_gb300.api import Grid
    from paper_1805_02144_gb300.inputs import balanced_state
    G = Grid(level)
    ng = G.ncells
    u0 = torch.from_numpy(balanced_state(G.cell_centres(), 3, 400.0)).cuda()
    res = {}
    from paper_1805_02144_gb300.api import SchemeState, exprb_step

    def replay_status(opts) -> dict:
        """The same 24 steps, untimed, with every step's device status and Krylov size."""
        st, u, codes, mmax = SchemeState(G), u0.clone(), [], 0
        for _ in range(24):
            u, info = exprb_step(G, "exprb53", 1800.0, u, state=st, opts=opts, stats=True)
            codes.append(info["status"])
            mmax = max(mmax, info["m_max_used"])
        bad = [k for k, c in enumerate(codes) if c != 0]
        return {"status": codes[bad[0]] if bad else 0, "steps_with_status": bad, "m_max_used": mmax}
    for name, opts in (("mixed", {"precision": 1, "tol": 1e-6}), ("fp64", {"tol": 1e-8})):
        timed_steps(G, u0, "exprb53", 1800.0, 2, opts, flush)          # warm-up
        ms, u, prof = timed_steps(G, u0, "exprb53", 1800.0, 24, opts, flush, profile=True)
        tot = sum(ms)
        res[name] = {"steps_per_s": 24 / (tot / 1e3), "ms_per_step": tot / 24, "tol": opts["tol"],
                     "phi_share": prof["phi_ms"] / tot, "state": u, **replay_status(opts)}
        if name == "mixed":
            gbs = prof["phi_bytes"] / (prof["phi_ms"] / 1e3) / 1e9
            hbm = _peaks().get("hbm_gbs", 6779.0)
            gbs_t = (prof["phi_bytes"] + prof["phi_table_bytes"]) / (prof["phi_ms"] / 1e3) / 1e9
            res[name]["roofline"] = {"kernel": "phi_kernel<float>", "bound": "hbm", "achieved": gbs,
                                     "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                                     "launch_ms": prof["phi_ms"] / max(prof["phi_launches"], 1),
                                     "with_tables": {"achieved": gbs_t, "frac": gbs_t / hbm,
                                                     "note": "vector bytes plus the FP32 operator "
                                                             "tables each pass streams"}}
    def rel(a, b):
        a, b = a.cpu().numpy(), b.cpu().numpy()
        return {"h": float(np.linalg.norm(a[3 * ng:] - b[3 * ng:]) / np.linalg.norm(b[3 * ng:])),
                "velocity": float(np.linalg.norm(a[:3 * ng] - b[:3 * ng]) / np.linalg.norm(b[:3 * ng]))}
    # the FP64 path at the mixed path's Krylov tolerance (untimed): separates
    # the FP32 rounding from the effect of the looser tolerance
    st, u = SchemeState(G), u0.clone()
    for _ in range(24):
        u = exprb_step(G, "exprb53", 1800.0, u, state=st, opts={"tol": 1e-6})
    um, uf = res["mixed"].pop("state"), res["fp64"].pop("state")
    return {"workload": f"exprb53, level-{level} grid ({ng} cells, n={4 * ng}), dt=1800 s, 12 h "
                        "(24 steps from the same seeded state, seed 3, 400 m)",
            "mixed": res["mixed"], "fp64": res["fp64"],
            "speedup_mixed_over_fp64": res["mixed"]["steps_per_s"] / res["fp64"]["steps_per_s"],
            "rel_l2_mixed_vs_fp64": rel(um, uf),
            "rel_l2_mixed_vs_fp64_same_tol": rel(um, u),
            "rel_l2_fp64_tol_1e-6_vs_1e-8": rel(u, uf),
            "note": "the FP64 path matches the FP64 oracle to 1e-10 (tests); mixed is within 1e-5"}


def batching_block() -> dict:
    """64-member exprb42 ensemble (levels 5/6/7, dt 900/1800/3600 s, 6 h) in one
    persistent launch replayed from a CUDA graph, against the same trajectories
    advanced one exprb_step at a time (the plain FP64 GPU form)."""
    import torch
    from paper_1805_02144_gb300.api import Ensemble, Grid, SchemeState, exprb_step
    from paper_1805_02144_gb300.inputs import balanced_state, ensemble_config
    cfg = ensemble_config()
    grids = {lev: Grid(lev) for lev in sorted({c["level"] for c in cfg})}
    gl = [grids[c["level"]] for c in cfg]
    u0 = [torch.from_numpy(balanced_state(g.cell_centres(), c["seed"], c["amplitude"])).cuda()
          for g, c in zip(gl, cfg)]
    E = Ensemble(gl, [c["dt"] for c in cfg], [c["nsteps"] for c in cfg], opts={"tol": TOL})

    def reset():
        for m, u in enumerate(u0):
            E.set_state(m, u)
        E.reset()

    # the launch before tuning: 96-thread blocks, one member per group, split by the work model
    reset()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    E.run()
    b.record()
    torch.cuda.synchronize()
    untuned_ms = a.elapsed_time(b)
    reset()
    t_tune = time.time()
    E.tune(rounds=4)
    tune_s = time.time() - t_tune

    reset()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            E.run(stream=s)
    torch.cuda.current_stream().wait_stream(s)
    times = []
    for rep in range(3):
        reset()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        g.replay()
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    st = E.stats()
    sh = E.shape()
    flop = E.work()
    ens_ms = min(times)
    member_steps = sum(c["nsteps"] for c in cfg)
    # the same trajectories one exprb_step call at a time
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for m, (G, c) in enumerate(zip(gl, cfg)):
        ss = SchemeState(G)
        u = u0[m].clone()
        out = torch.empty_like(u)
        for _ in range(c["nsteps"]):
            exprb_step(G, "exprb42", c["dt"], u, out=out, state=ss, opts={"tol": TOL})
            u, out = out, u
    b.record()
    torch.cuda.synchronize()
    seq_ms = a.elapsed_time(b)
    mm = st["member_ms"]
    gms = {}
    for m, g in enumerate(sh["member_group"]):   # a group runs its members one after the other
        gms[g] = gms.get(g, 0.0) + mm[m]
    gl_ms = list(gms.values())
    achieved = flop / (ens_ms / 1e3) / 1e12
    return {"workload": "64 exprb42 members (seed 4): levels 5/6/7, dt 900/1800/3600 s, amplitudes "
                        "U[50,400] m, 6 h each (804 member-steps), FP64, Tol 1e-8",
            "ensemble_ms": ens_ms, "member_steps_per_s": member_steps / (ens_ms / 1e3),
            "untuned_ms": untuned_ms, "tune_s": tune_s,
            "sequential_ms": seq_ms, "sequential_member_steps_per_s": member_steps / (seq_ms / 1e3),
            "speedup_over_sequential": seq_ms / ens_ms,
            "launch": "one cooperative launch per 6 h run, replayed from a CUDA graph",
            "tuned_shape": {"threads": sh["threads"], "blocks_per_sm": sh["blocks_per_sm"],
                            "blocks": sh["nblocks"], "groups": sh["groups"],
                            "stacked_members": len(mm) - sh["groups"]},
            "group_ms_max": max(gl_ms), "group_ms_mean": sum(gl_ms) / len(gl_ms),
            "member_ms_mean": sum(mm) / len(mm),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP64_PEAK_TFLOPS,
                         "note": "algorithmic FP64 operations of all members / ensemble time"},
            "blocks_per_group": {"min": min(st["blocks"]), "max": max(st["blocks"]),
                                 "total": sh["nblocks"]}}


def schemes_block(flush) -> dict:
    """The other schemes of the comparison on the level-7 headline grid (FP64,
    Tol 1e-8, seed 2): exprb42 / pexprb43 / exprb53 at dt 3600 s (24 steps) and
    epi3 at dt 900 s (96 steps), per-step CUDA events, L2 flushed between steps."""
    import torch
    from paper_1805_02144_gb300.api import Grid, SchemeState
    from paper_1805_02144_gb300.inputs import balanced_state
    G = Grid(LEVEL)
    u0 = torch.from_numpy(balanced_state(G.cell_centres(), SEED, AMP)).cuda()
    out = {}
    for scheme, dt, n in (("exprb42", 3600.0, 24), ("pexprb43", 3600.0, 24), ("exprb53", 3600.0, 24),
                          ("epi3", 900.0, 96)):
        st = SchemeState(G)
        ms, u, _ = timed_steps(G, u0, scheme, dt, n, {"tol": TOL}, flush, state=st)
        tot = sum(ms)
        out[scheme] = {"dt": dt, "steps": n, "steps_per_s": n / (tot / 1e3),
                       "simulated_hours_per_s": n * dt / 3600.0 / (tot / 1e3),
                       "finite": bool(torch.isfinite(u).all().item())}
    return {"workload": "level-7 grid, FP64, Tol 1e-8, seed 2 (400 m); 24 h simulated per scheme", **out}


def efficiency_block(level: int = 5) -> dict:
    """Error against run time, the methodology of the paper's efficiency
    tables, on the synthetic state: a 6 h integration on a level-5 grid from
    the seeded balanced state (seed 2, 400 m), each scheme at dt in
    {900, 1800, 3600} s and Tol in {1e-6, 1e-8, 1e-10}; error = relative L2 of
    h at 6 h against exprb53 with dt = 225 s and Tol = 1e-12."""
    import time
    import torch
    from paper_1805_02144_gb300.api import Grid, SchemeState, exprb_step
    from paper_1805_02144_gb300.inputs import balanced_state
    G = Grid(level)
    ng = G.ncells
    u0 = torch.from_numpy(balanced_state(G.cell_centres(), SEED, AMP)).cuda()
    T = 6 * 3600.0

    def run(scheme, dt, tol):
        st = SchemeState(G)
        u = u0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(int(round(T / dt))):
            u, info = exprb_step(G, scheme, dt, u, state=st, opts={"tol": tol}, stats=True)
            if info["status"] != 0:
                return None, info["status"], time.perf_counter() - t0
        torch.cuda.synchronize()
        return u, 0, time.perf_counter() - t0

    ref, _, _ = run("exprb53", 225.0, 1e-12)
    href = ref[3 * ng:]
    rows = []
    for scheme in ("exprb42", "pexprb43", "exprb53", "epi3"):
        for dt in (900.0, 1800.0, 3600.0):
            for tol in (1e-6, 1e-8, 1e-10):
                u, st, wall = run(scheme, dt, tol)
                err = None if u is None else float(torch.linalg.norm(u[3 * ng:] - href) / torch.linalg.norm(href))
                rows.append({"scheme": scheme, "dt": dt, "tol": tol, "rel_err_h": err, "ms": 1e3 * wall,
                             "status": st})
    return {"workload": f"level-{level} grid ({ng} cells), 6 h from the seeded balanced state (seed 2, "
                        "400 m), FP64; reference exprb53 dt 225 s Tol 1e-12; wall time per run with host "
                        "status checks each step", "runs": rows}


def conservation_block(levels=(6, 4), cap_s: float = 60.0) -> dict:
    """15 simulated days on the paper's level-6 grid (and on level 4) from the
    seeded balanced state (seed 2), FP64, Tol 1e-8, with the step sizes of the
    paper's conservation runs (exprb53 6 h, exprb42 and pexprb43 4.8 h, epi3
    2 h): normalised drift (X(t) - X(0)) / X(0) of total mass, energy and
    potential enstrophy.  A scheme that fails (the trajectory can go unstable
    at these step sizes) or that would take more than cap_s seconds stops
    early and says so."""
    out = {f"level{lev}": conservation_run(lev, cap_s) for lev in levels}
    out["level6_gamma_h_1.25e-2"] = conservation_run(6, cap_s, gamma_h=1.25e-2)
    return out


def conservation_run(level: int, cap_s: float, gamma_h: float = None) -> dict:
    import time
    import torch
    from paper_1805_02144_gb300.api import Grid, SchemeState, exprb_step, swe_diagnostics
    from paper_1805_02144_gb300.inputs import balanced_state
    G = Grid(level) if gamma_h is None else Grid(level, gamma_h=gamma_h)
    u0 = torch.from_numpy(balanced_state(G.cell_centres(), SEED, AMP)).cuda()
    d0 = swe_diagnostics(G, u0)
    out = {}
    for scheme, hours in (("exprb53", 6.0), ("exprb42", 4.8), ("pexprb43", 4.8), ("epi3", 2.0)):
        dt = hours * 3600.0
        n = int(round(15 * 24 / hours))
        st = SchemeState(G)
        u, d = u0, d0
        worst = {k: 0.0 for k in d0}
        status = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        done = 0
        for _ in range(n):
            un, info = exprb_step(G, scheme, dt, u, state=st, opts={"tol": TOL}, stats=True)
            if info["status"] != 0:
                status = info["status"]
                break
            u = un
            d = swe_diagnostics(G, u)
            done += 1
            for k in d0:
                worst[k] = max(worst[k], abs(d[k] - d0[k]) / abs(d0[k]))
            if time.perf_counter() - t0 > cap_s:
                break
        wall = time.perf_counter() - t0
        out[scheme] = {"dt_hours": hours, "steps": done, "days": done * hours / 24.0, "wall_s": wall,
                       "status": status, "drift_end": {k: (d[k] - d0[k]) / d0[k] for k in d0},
                       "max_abs_drift": worst}
    gh = f", gamma_h = {gamma_h:g}" if gamma_h is not None else ""
    return {"workload": f"level-{level} grid ({G.ncells} cells){gh}, 15 days from the seeded balanced state "
                        "(seed 2, 400 m), FP64, Tol 1e-8; diagnostics after every step", **out}


def adjoint_block(flush) -> dict:
    """Gradient of the 6 h exprb42 forecast misfit (level 6, dt 1800 s, 12 steps,
    Tol 1e-10; observations: the 6 h truth forecast from seed 5 at 1000 seeded
    cells plus N(0, 5^2); first guess: seed 6) by per-step checkpoints,
    recomputation with a Krylov tape and the reverse sweep, against the
    forecast itself; 8 frozen-decision central differences as a check."""
    import torch
    from paper_1805_02144_gb300.api import Grid, SchemeState, exprb_step, exprb_step_adjoint
    from paper_1805_02144_gb300.inputs import balanced_state, fd_directions, observation_network
    G = Grid(6)
    x = G.cell_centres()
    ng = G.ncells
    dt, nsteps, tol = 1800.0, 12, 1e-10
    opts = {"tol": tol}

    def forecast(u, trace: bool):
        st = SchemeState(G)
        states, traces = [u], []
        for _ in range(nsteps):
            if trace:
                u, info = exprb_step(G, "exprb42", dt, u, state=st, opts=opts, stats=True, trace_cap=4096)
                traces.append(info["trace"])
            else:
                u = exprb_step(G, "exprb42", dt, u, state=st, opts=opts)
            states.append(u)
        return states, traces

    truth, _ = forecast(torch.from_numpy(balanced_state(x, 5, 400.0)).cuda(), False)
    cells, y, sigma = observation_network(x, 1000, 7, 5.0, h_truth=truth[-1][3 * ng:].cpu().numpy())
    cells_t = torch.from_numpy(cells).cuda()
    y_t = torch.from_numpy(y).cuda()
    u0 = torch.from_numpy(balanced_state(x, 6, 400.0)).cuda()

    def misfit(u):
        r = (u[3 * ng:][cells_t] - y_t) / sigma
        lam = torch.zeros_like(u)
        lam.index_add_(0, 3 * ng + cells_t, r / sigma)
        return 0.5 * float(torch.dot(r, r)), lam

    def gradient(states, traces):
        J, lam = misfit(states[-1])
        for k in reversed(range(nsteps)):
            lam = exprb_step_adjoint(G, "exprb42", dt, states[k], traces[k], lam, opts=opts)
        return J, lam

    def timed(fn, reps=3):
        best, out = None, None
        for rep in range(reps):
            flush.fill_(float(rep))  # 256 MB write: L2 (129 MB) holds nothing of the last run
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            out = fn()
            b.record()
            torch.cuda.synchronize()
            t = a.elapsed_time(b)
            best = t if best is None else min(best, t)
        return best, out

    states, traces = forecast(u0, True)
    gradient(states, traces)
    fwd_ms, _ = timed(lambda: forecast(u0, False))
    fwdt_ms, (states, traces) = timed(lambda: forecast(u0, True))
    adj_ms, (J, g) = timed(lambda: gradient(states, traces))
    rp = [{"tol": tol, "replay": [[r["tau"], r["m"], float(r["accepted"])] for r in tr]} for tr in traces]

    def J_replayed(u):
        st = SchemeState(G)
        for k in range(nsteps):
            u = exprb_step(G, "exprb42", dt, u, state=st, opts=rp[k])
        return misfit(u)[0]

    worst = 0.0
    for d, eps in fd_directions(u0.cpu().numpy(), 8, 11):
        dd = torch.from_numpy(d).cuda()
        fd = (J_replayed(u0 + eps * dd) - J_replayed(u0 - eps * dd)) / (2 * eps)
        worst = max(worst, abs(fd - float(torch.dot(g, dd))) / abs(fd))
    return {"workload": "gradient of 0.5 sum (h - y)^2 / sigma^2 at 1000 seeded cells (sigma 5 m, y = 6 h "
                        "truth forecast from seed 5 plus noise) after a 6 h exprb42 forecast from seed 6: "
                        "level-6 grid (40962 cells), dt 1800 s, 12 steps, FP64, Tol 1e-10, frozen substep "
                        "decisions, per-step checkpoints with recomputation",
            "forecast_ms": fwd_ms, "forecast_with_trace_ms": fwdt_ms, "gradient_ms": adj_ms,
            "adjoint_over_forward": adj_ms / fwd_ms, "misfit": J,
            "fd_check": {"directions": 8, "eps": "1e-6 ||u0|| / ||d||", "max_rel_diff": worst},
            "attempts_per_step": [len(t) for t in traces]}


def gpu_arm(args) -> None:
    import torch
    from paper_1805_02144_gb300.ranks import from_env, job_rate, max_over_ranks
    rk = from_env()
    world, rank, local = rk.world, rk.rank, rk.local
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1805_02144_gb300 import build
    build.build()
    from paper_1805_02144_gb300.api import Grid, SchemeState, exprb_step
    from paper_1805_02144_gb300.inputs import balanced_state

    G = Grid(LEVEL)
    u0 = torch.from_numpy(balanced_state(G.cell_centres(), SEED, AMP)).cuda()
    st = SchemeState(G)
    opts = {"tol": TOL}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    sampler = ClockSampler(local)
    _, uw, _ = timed_steps(G, u0, SCHEME, DT, args.warmup, opts, flush, state=st)
    if dist:
        dist.barrier()
    ms, ucur, prof = timed_steps(G, uw, SCHEME, DT, args.steps, opts, flush, state=st, profile=True)
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    t_ms = max_over_ranks(sum(ms), dist, "cuda")
    value = job_rate(world, args.steps, t_ms)

    # end to end through the public API: pinned host state in, host state out,
    # over the same steps as the timed loop (the same warm-up from u0 with a
    # fresh scheme state, so every step does the same work)
    n = G.n
    st = SchemeState(G)
    _, uw_e2e, _ = timed_steps(G, u0, SCHEME, DT, args.warmup, opts, flush, state=st)
    h_in = torch.empty(n, dtype=torch.float64, pin_memory=True)
    h_in.copy_(uw_e2e.cpu())
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
    e_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev2), dist, "cuda")
    e2e = job_rate(world, args.steps, e_ms)
    finite = bool(torch.isfinite(ucur).all().item())

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
            "hbm_gbs_with_tables": (prof["phi_bytes"] + prof["phi_table_bytes"]) / (prof["phi_ms"] / 1e3) / 1e9,
            "iom2_iterations_per_step": prof["iom2_iterations"] / args.steps,
            # per cell: the kernel's FP64 operation count of one IOM2 column (346) and the
            # fewest operations Algorithm 1 needs for it: J x of Eqs. eq:dynja-eq:dynjc
            # in factored form (288), two window dots (16), the orthogonalisation (16)
            # and the norm (8); frac_minimal rates the kernel by the latter
            "flop_per_cell_iom2_column": {"kernel": 346, "minimal": 328},
            "frac_minimal": achieved * 328.0 / 346.0 / FP64_PEAK_TFLOPS,
            "phase_ms_per_step": {k: v / args.steps for k, v in prof["phase_ms"].items()},
        },
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n},
        "gpu_launches": prof["kernel_launches"],
        "clocks": clocks,
        "finite": finite,
    }
    if world == 1 and not args.no_extra:
        line["precision"] = precision_block(flush)
        line["batching"] = batching_block()
        line["adjoint"] = adjoint_block(flush)
        line["schemes"] = schemes_block(flush)
        line["conservation"] = conservation_block()
        line["efficiency"] = efficiency_block()
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
        try:  # every host core: one independent oracle process per core
            ncore = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
            res = oracle_replicas(ncore)
            line["cpu_baseline_all_cores"] = {
                "value": res["value"], "unit": UNIT, "cores": ncore, "kind": "oracle",
                "sample": f"{ncore} independent oracle processes (one thread each), one {SCHEME} step of "
                          "the same level-7 workload each, started together; value = steps over the "
                          "span from the first start to the last end",
                "step_s_min_max": [min(res["step_s"]), max(res["step_s"])]}
        except Exception as e:
            line["cpu_baseline_all_cores"] = {"value": None, "unit": UNIT, "kind": "oracle",
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
    ap.add_argument("--no-extra", action="store_true", help="skip the precision/batching/adjoint blocks")
    ap.add_argument("--only", choices=["precision", "batching", "adjoint", "schemes", "conservation",
                                       "efficiency"],
                    help="run one extra block alone and print it (for profiling)")
    args = ap.parse_args()
    if args.only:
        import torch
        from paper_1805_02144_gb300 import build
        build.build()
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        fn = {"precision": lambda: precision_block(flush), "batching": batching_block,
              "adjoint": lambda: adjoint_block(flush), "schemes": lambda: schemes_block(flush),
              "conservation": conservation_block, "efficiency": efficiency_block}[args.only]
        print(json.dumps({args.only: fn()}), flush=True)
        return
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
