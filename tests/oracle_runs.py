"""Oracle trajectories run in worker processes for the long GPU parity tests.

A level-7 oracle trajectory takes a minute or more of host time, so the long
parity tests start them in spawned worker processes (never forked: the parent
holds a CUDA context) and run the GPU side meanwhile.  Each worker builds its
own oracle grid and returns plain arrays: the final state in the oracle's
cell order, and per step the decisions [tau, m, accepted] of every attempt of
every phi call, in call order (the record layout the library's replay option
takes), with the per-step Krylov product counts.
"""
import os


def trajectory(scheme: str, level: int, seed: int, amp: float, dt: float, nsteps: int, tol: float):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle.phipm import PhiOpts
    from oracle.schemes import KrylovPhi, step
    from oracle.swe import make_swe
    from paper_1805_02144_gb300.inputs import balanced_state
    s = make_swe(level)
    u = balanced_state(s.grid.x, seed, amp)
    kp = KrylovPhi(s, PhiOpts(tol=tol))
    decisions, njv = [], []
    u_prev = None
    for _ in range(nsteps):
        k0 = len(kp.stats)
        u_next = step(scheme, s, u, dt, kp, u_prev=u_prev)
        calls = kp.stats[k0:]
        decisions.append([[a.tau, a.m, 1.0 if a.accepted else 0.0] for _, st in calls for a in st.trace])
        njv.append(sum(st.n_jv for _, st in calls))
        if scheme == "epi3":
            u_prev = u
        u = u_next
    return u, decisions, njv


def diagnostics_run(scheme: str, level: int, seed: int, amp: float, dt: float, nsteps: int, tol: float,
                    gamma_h: float):
    """The oracle trajectory of ``scheme`` with the conservation diagnostics
    (total mass, energy, potential enstrophy) of the state after every step."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle.phipm import PhiOpts
    from oracle.schemes import KrylovPhi, step
    from oracle.swe import make_swe
    from paper_1805_02144_gb300.inputs import balanced_state
    s = make_swe(level, gamma_h=gamma_h)
    u = balanced_state(s.grid.x, seed, amp)
    kp = KrylovPhi(s, PhiOpts(tol=tol))
    diag = [(s.mass(u), s.energy(u), s.potential_enstrophy(u))]
    u_prev = None
    for _ in range(nsteps):
        u_next = step(scheme, s, u, dt, kp, u_prev=u_prev)
        if scheme == "epi3":
            u_prev = u
        u = u_next
        diag.append((s.mass(u), s.energy(u), s.potential_enstrophy(u)))
    return u, diag
