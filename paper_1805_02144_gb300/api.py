"""Python surface over the C ABI, with the same names (torch tensors in, out).

Vectors are torch float64 CUDA tensors of n = 4 * ncells elements in the
grid's cell order; work is enqueued on the current torch CUDA stream unless a
stream is given.  Nothing here computes: each function checks arguments,
passes device pointers to libswe_exprb.so and raises on a nonzero status.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib
from ._lib import PhiAttemptC, PhiStatsC, SCHEMES, check, default_opts, load

EARTH_RADIUS = 6.37122e6
GRAVITY = 9.80616
OMEGA = 7.292e-5
GAMMA_H = 0.04e-2


def _stream(stream) -> C.c_void_p:
    if stream is None:
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _ptr(t: Optional[torch.Tensor], n: int, name: str) -> C.c_void_p:
    if t is None:
        return C.c_void_p(0)
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError(f"{name} must be a CUDA float64 tensor")
    if not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{name} must be contiguous with {n} elements")
    return C.c_void_p(t.data_ptr())


class Grid:
    """Handle of swe_create_grid (icosahedral geodesic grid + operator tables)."""

    def __init__(self, level: int, radius: float = EARTH_RADIUS, g: float = GRAVITY,
                 omega: float = OMEGA, gamma_h: float = GAMMA_H, reorder: bool = True,
                 host_only: bool = False):
        L = load()
        h = C.c_void_p()
        create = L.swe_create_grid_host if host_only else L.swe_create_grid
        check(create(level, radius, g, omega, gamma_h, int(reorder), C.byref(h)))
        self.handle = h
        self.level = level
        nc, n, nA, nu = C.c_int64(), C.c_int64(), C.c_int64(), C.c_double()
        check(L.swe_grid_query(h, C.byref(nc), C.byref(n), C.byref(nA), C.byref(nu)))
        self.ncells, self.n, self.nA, self.nu = nc.value, n.value, nA.value, nu.value

    def cell_centres(self) -> np.ndarray:
        out = np.empty(3 * self.ncells)
        check(load().swe_grid_cell_centres(self.handle, out.ctypes.data_as(C.POINTER(C.c_double))))
        return out.reshape(3, self.ncells).T.copy()

    def cell_areas(self) -> np.ndarray:
        out = np.empty(self.ncells)
        check(load().swe_grid_cell_areas(self.handle, out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def export(self, table: str) -> np.ndarray:
        """Host copy of an operator table (see swe_grid_export), shaped [..., ncells]."""
        ng = self.ncells
        shapes = {"nbr": (6, ng), "gen": (ng,), "wl": (6, ng), "wld": (ng,), "nc": (3, 6, ng), "ndd": (3, ng),
                  "sdg": (3, ng), "vc": (3, 6, ng), "vd": (3, ng), "wlT": (6, ng), "ncT": (3, 6, ng),
                  "vcT": (3, 6, ng)}
        out = np.empty(shapes[table], dtype=np.int32 if table in ("nbr", "gen") else np.float64)
        check(load().swe_grid_export(self.handle, table.encode(), out.ctypes.data_as(C.c_void_p),
                                     out.size))
        return out

    def close(self) -> None:
        if self.handle:
            load().swe_destroy_grid(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def swe_create_grid(level: int, **kw) -> Grid:
    return Grid(level, **kw)


def _new(grid: Grid, like: Optional[torch.Tensor] = None) -> torch.Tensor:
    dev = like.device if like is not None else torch.device("cuda")
    return torch.empty(grid.n, dtype=torch.float64, device=dev)


def swe_rhs(grid: Grid, u: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    out = _new(grid, u) if out is None else out
    check(load().swe_rhs(grid.handle, _ptr(u, grid.n, "u"), _ptr(out, grid.n, "out"), _stream(stream)))
    return out


def swe_jv(grid: Grid, u: torch.Tensor, x: torch.Tensor, out: Optional[torch.Tensor] = None,
           stream=None) -> torch.Tensor:
    out = _new(grid, u) if out is None else out
    check(load().swe_jv(grid.handle, _ptr(u, grid.n, "u"), _ptr(x, grid.n, "x"),
                        _ptr(out, grid.n, "out"), _stream(stream)))
    return out


def swe_grid_set_topography(grid: Grid, hs: Optional[np.ndarray]) -> None:
    """Set (or, with None, remove) the surface height h_s [m] per cell (grid order)."""
    if hs is None:
        check(load().swe_grid_set_topography(grid.handle, None))
        return
    a = np.ascontiguousarray(np.asarray(hs, dtype=np.float64))
    if a.size != grid.ncells:
        raise ValueError("hs needs one value per cell")
    check(load().swe_grid_set_topography(grid.handle, a.ctypes.data_as(C.POINTER(C.c_double))))


def swe_diagnostics(grid: Grid, u: torch.Tensor, stream=None) -> dict:
    """Total mass, energy and potential enstrophy of a state (see the header)."""
    out = np.zeros(3)
    check(load().swe_diagnostics(grid.handle, _ptr(u, grid.n, "u"), out.ctypes.data_as(C.POINTER(C.c_double)),
                                 _stream(stream)))
    return {"mass": float(out[0]), "energy": float(out[1]), "potential_enstrophy": float(out[2])}


def swe_jtv(grid: Grid, u: torch.Tensor, lam: torch.Tensor, out: Optional[torch.Tensor] = None,
            stream=None) -> torch.Tensor:
    """out = J(u)^T lam (transpose of the Jacobian of Eqs. (eq:dynja)-(eq:dynjc))."""
    out = _new(grid, u) if out is None else out
    check(load().swe_jtv(grid.handle, _ptr(u, grid.n, "u"), _ptr(lam, grid.n, "lam"),
                         _ptr(out, grid.n, "out"), _stream(stream)))
    return out


def swe_dqtv(grid: Grid, x: torch.Tensor, lam: torch.Tensor, out: Optional[torch.Tensor] = None,
             stream=None) -> torch.Tensor:
    """out = (J(x) - J(0))^T lam (transposed derivative of the quadratic part of F at x)."""
    out = _new(grid, x) if out is None else out
    check(load().swe_dqtv(grid.handle, _ptr(x, grid.n, "x"), _ptr(lam, grid.n, "lam"),
                          _ptr(out, grid.n, "out"), _stream(stream)))
    return out


def _opts(opts) -> tuple[_lib.PhiOptsC, object]:
    """Build a phi_opts struct from a dict; returns (struct, keep-alive)."""
    if opts is None:
        return default_opts(), None
    if isinstance(opts, _lib.PhiOptsC):
        return opts, None
    o = default_opts(**{k: v for k, v in opts.items() if k != "replay"})
    keep = None
    if opts.get("replay") is not None:
        rec = np.ascontiguousarray(np.asarray(opts["replay"], dtype=np.float64).reshape(-1, 3))
        keep = rec
        o.replay = rec.ctypes.data_as(C.POINTER(C.c_double))
        o.n_replay = rec.shape[0]
    return o, keep


def _stats(trace_cap: int) -> tuple[PhiStatsC, object]:
    st = PhiStatsC()
    buf = None
    if trace_cap > 0:
        buf = (PhiAttemptC * trace_cap)()
        st.trace = C.cast(buf, C.POINTER(PhiAttemptC))
        st.trace_cap = trace_cap
    return st, buf


def _stats_dict(st: PhiStatsC) -> dict:
    d = {k: getattr(st, k) for k in ("n_jv", "n_substeps", "n_reject", "m_last", "m_max_used", "status")}
    d["trace"] = [dict(t=st.trace[i].t, tau=st.trace[i].tau, omega=st.trace[i].omega, m=st.trace[i].m,
                       accepted=bool(st.trace[i].accepted), call=st.trace[i].call)
                  for i in range(st.n_trace)]
    return d


def phi_action(grid: Grid, u_lin: torch.Tensor, dt: float, v: Sequence[Optional[torch.Tensor]],
               rho: Sequence[float], out: Optional[Sequence[torch.Tensor]] = None, opts=None,
               stats: bool = False, trace_cap: int = 0, stream=None):
    """[sum_l rho_i^l phi_l(rho_i dt J(u_lin)) v_l for rho_i in rho] (Algorithm 1)."""
    p = len(v) - 1
    ns = len(rho)
    outs = [_new(grid, u_lin) for _ in range(ns)] if out is None else list(out)
    vp = (C.c_void_p * (p + 1))(*[_ptr(x, grid.n, f"v[{i}]") for i, x in enumerate(v)])
    yp = (C.c_void_p * ns)(*[_ptr(y, grid.n, f"out[{i}]") for i, y in enumerate(outs)])
    rh = (C.c_double * ns)(*[float(r) for r in rho])
    o, keep = _opts(opts)
    st, buf = _stats(trace_cap) if (stats or trace_cap) else (None, None)
    check(load().phi_action(grid.handle, _ptr(u_lin, grid.n, "u_lin"), float(dt), p, vp, ns, rh, yp,
                            C.byref(o), C.byref(st) if st is not None else None, _stream(stream)))
    del keep, buf
    return (outs, _stats_dict(st)) if st is not None else outs


class SchemeState:
    """swe_scheme_state: epi3 history and the Krylov size carried per call slot."""

    def __init__(self, grid: Grid):
        h = C.c_void_p()
        check(load().swe_scheme_state_create(grid.handle, C.byref(h)))
        self.handle = h
        self.grid = grid

    def reset(self) -> None:
        check(load().swe_scheme_state_reset(self.handle))

    def close(self) -> None:
        if self.handle:
            load().swe_scheme_state_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def exprb_step(grid: Grid, scheme: str, dt: float, u_n: torch.Tensor,
               out: Optional[torch.Tensor] = None, state: Optional[SchemeState] = None, opts=None,
               stats: bool = False, trace_cap: int = 0, stream=None):
    """One step u_{n+1} of scheme in {epi2, exprb42, pexprb43, exprb53, epi3}."""
    out = _new(grid, u_n) if out is None else out
    if state is None:
        raise ValueError("exprb_step needs a SchemeState (epi3 history, Krylov size carry)")
    o, keep = _opts(opts)
    st, buf = _stats(trace_cap) if (stats or trace_cap) else (None, None)
    check(load().exprb_step(grid.handle, SCHEMES[scheme], float(dt), _ptr(u_n, grid.n, "u_n"),
                            _ptr(out, grid.n, "out"), state.handle, C.byref(o),
                            C.byref(st) if st is not None else None, _stream(stream)))
    del keep, buf
    return (out, _stats_dict(st)) if st is not None else out


def _trace_array(trace) -> tuple:
    """phi_attempt array from exprb_step's stats["trace"] (list of dicts)."""
    arr = (PhiAttemptC * len(trace))()
    for i, r in enumerate(trace):
        arr[i].t = float(r["t"])
        arr[i].tau = float(r["tau"])
        arr[i].omega = float(r.get("omega", 0.0))
        arr[i].m = int(r["m"])
        arr[i].accepted = int(bool(r["accepted"]))
        arr[i].call = int(r["call"])
    return arr


def exprb_step_adjoint(grid: Grid, scheme: str, dt: float, u_n: torch.Tensor, trace, lam_np1: torch.Tensor,
                       out: Optional[torch.Tensor] = None, opts=None, stats: bool = False, stream=None):
    """lam_n = (d u_{n+1}/d u_n)^T lam_np1 with the decisions of ``trace`` frozen
    (``trace``: exprb_step's stats["trace"] for the step from u_n)."""
    if not trace:
        raise ValueError("exprb_step_adjoint needs the forward step's trace")
    out = _new(grid, u_n) if out is None else out
    o, keep = _opts(opts)
    arr = _trace_array(trace)
    st = PhiStatsC() if stats else None
    check(load().exprb_step_adjoint(grid.handle, SCHEMES[scheme], float(dt), _ptr(u_n, grid.n, "u_n"), arr,
                                    len(trace), _ptr(lam_np1, grid.n, "lam_np1"), _ptr(out, grid.n, "out"),
                                    C.byref(o), C.byref(st) if st is not None else None, _stream(stream)))
    del keep
    return (out, _stats_dict(st)) if st is not None else out


class ExprbStepFunction(torch.autograd.Function):
    """u_{n+1} = exprb_step(u_n) with backward = exprb_step_adjoint (frozen decisions).

    The input u_n is the checkpoint; backward recomputes the step from it."""

    @staticmethod
    def forward(ctx, u_n, grid, scheme, dt, state, opts, trace_cap):
        out, st = exprb_step(grid, scheme, dt, u_n.detach(), state=state, opts=opts, stats=True,
                             trace_cap=trace_cap)
        if st["status"] != 0:
            raise RuntimeError(f"exprb_step failed on the device: status {st['status']}")
        if len(st["trace"]) >= trace_cap:
            raise RuntimeError("trace_cap too small for the step's attempts")
        ctx.save_for_backward(u_n.detach())
        ctx.meta = (grid, scheme, dt, st["trace"], opts)
        return out

    @staticmethod
    def backward(ctx, g):
        (u_n,) = ctx.saved_tensors
        grid, scheme, dt, trace, opts = ctx.meta
        lam = exprb_step_adjoint(grid, scheme, dt, u_n, trace, g.contiguous(), opts=opts)
        return lam, None, None, None, None, None, None


def exprb_step_differentiable(grid: Grid, scheme: str, dt: float, u_n: torch.Tensor, state: "SchemeState",
                              opts=None, trace_cap: int = 4096) -> torch.Tensor:
    """exprb_step as a torch autograd node (EPI2, exprb42, pexprb43, exprb53)."""
    return ExprbStepFunction.apply(u_n, grid, scheme, dt, state, opts, trace_cap)


def swe_selftest_wait(limit_s: float = 0.02, preset_abort: int = 0, stream=None) -> int:
    """Run the bounded device-side wait on a flag that nothing sets; returns the
    abort word it left (SWE_ERR_TIMEOUT, or preset_abort if one was given)."""
    st = C.c_int(0)
    check(load().swe_selftest_wait(int(limit_s * 1e9), int(preset_abort), C.byref(st), _stream(stream)))
    return st.value


def swe_device_status(grid: Grid, stream=None) -> None:
    check(load().swe_device_status(grid.handle, _stream(stream)))


def swe_profile_enable(grid: Grid, on: bool = True) -> None:
    check(load().swe_profile_enable(grid.handle, int(on)))


def swe_profile_read(grid: Grid, stream=None) -> dict:
    pr = _lib.ProfileC()
    check(load().swe_profile_read(grid.handle, C.byref(pr), _stream(stream)))
    d = {k: getattr(pr, k) for k, _ in _lib.ProfileC._fields_ if k != "phase_ms"}
    names = ["prologue", "w_pass1", "w_pass2", "iom2_pass1", "iom2_pass2_dots", "orth_pass1_norm",
             "decide_tail", "combine", "taylor", "decide_head"]
    d["phase_ms"] = {n: pr.phase_ms[i] for i, n in enumerate(names)}
    return d


class Ensemble:
    """swe_ensemble: independent exprb42 trajectories advanced by one persistent launch."""

    def __init__(self, grids: Sequence[Grid], dt: Sequence[float], nsteps: Sequence[int], opts=None):
        L = load()
        nm = len(grids)
        gh = (C.c_void_p * nm)(*[g.handle for g in grids])
        dts = (C.c_double * nm)(*[float(x) for x in dt])
        ns = (C.c_int * nm)(*[int(x) for x in nsteps])
        o, keep = _opts(opts)
        h = C.c_void_p()
        check(L.swe_ensemble_create(gh, nm, dts, ns, C.byref(o), C.byref(h)))
        del keep
        self.handle = h
        self.grids = list(grids)
        self.nmem = nm

    def set_state(self, m: int, u: torch.Tensor, stream=None) -> None:
        check(load().swe_ensemble_set_state(self.handle, m, _ptr(u, self.grids[m].n, "u"), _stream(stream)))

    def get_state(self, m: int, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        out = _new(self.grids[m]) if out is None else out
        check(load().swe_ensemble_get_state(self.handle, m, _ptr(out, self.grids[m].n, "out"), _stream(stream)))
        return out

    def run(self, stream=None) -> None:
        check(load().swe_ensemble_run(self.handle, _stream(stream)))

    def reset(self, stream=None) -> None:
        """Forget the Krylov sizes carried from earlier steps (new trajectories)."""
        check(load().swe_ensemble_reset(self.handle, _stream(stream)))

    def tune(self, rounds: int = 2, stream=None) -> None:
        check(load().swe_ensemble_tune(self.handle, rounds, _stream(stream)))

    def stats(self, stream=None) -> dict:
        nm = self.nmem
        st = (PhiStatsC * nm)()
        ms = (C.c_double * nm)()
        nb = (C.c_int * nm)()
        check(load().swe_ensemble_stats(self.handle, st, ms, nb, _stream(stream)))
        return {"status": [st[i].status for i in range(nm)], "n_jv": [st[i].n_jv for i in range(nm)],
                "member_ms": [ms[i] for i in range(nm)], "blocks": [nb[i] for i in range(nm)]}

    def shape(self) -> dict:
        """The launch in use: threads per block, blocks per SM, blocks launched,
        number of member groups and each member's group."""
        t, per, nb, ng = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        mg = (C.c_int * self.nmem)()
        check(load().swe_ensemble_shape(self.handle, C.byref(t), C.byref(per), C.byref(nb), C.byref(ng), mg))
        return {"threads": t.value, "blocks_per_sm": per.value, "nblocks": nb.value, "groups": ng.value,
                "member_group": [mg[i] for i in range(self.nmem)]}

    def work(self, stream=None) -> float:
        """Algorithmic FP64 operations of the last run."""
        f = C.c_double()
        check(load().swe_ensemble_work(self.handle, C.byref(f), _stream(stream)))
        return f.value

    def close(self) -> None:
        if self.handle:
            load().swe_ensemble_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
