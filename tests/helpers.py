"""Helpers shared by the parity tests: run a workload through the FP64 oracle
and through the CUDA library (the C ABI via its ctypes binding), and compare."""
from __future__ import annotations

import numpy as np


def run_oracle(oracle_mod, wl, steps, links_edit=None, bcs=None):
    nt, links = oracle_mod.geometry(**wl.geometry_args())
    if links_edit is not None:
        links = links_edit(links)
    o = oracle_mod.Oracle(nt, links, wl.bcs if bcs is None else bcs, lam=wl.lam, mu=wl.mu,
                          rho0=wl.rho0, tau=wl.tau, wall_node=wl.wall_node)
    o.step(steps)
    F = o.fields()
    return {"u": F["u"], "v": F["v"], "sigma": F["sigma"], "mask": nt.astype(bool)}


def run_gpu(wl, steps, storage="f32", links_edit=None, bcs=None, chunks=None, time_block=0,
            in_place=False):
    from paper_2208_04088_gb300 import _native as N
    nt, links = N.lbm_geom_build(**wl.geometry_args())
    if links_edit is not None:
        links = links_edit(links)
    d = N.Desc(nt, links, wl.bcs if bcs is None else bcs, wl.lam, wl.mu, wl.rho0, tau=wl.tau,
               storage=storage, wall_node=wl.wall_node, time_block=time_block, in_place=in_place)
    s = N.Solver(d)
    if chunks is None:
        s.step(steps)
    else:
        for c in chunks:
            s.step(c)
    s.sync()
    F = s.fields_host()
    info = s.info()
    s.close()
    F["mask"] = nt.astype(bool)
    F["info"] = info
    return F


def rel_l2(a, b, mask):
    a = np.asarray(a, dtype=np.float64)[..., mask]
    b = np.asarray(b, dtype=np.float64)[..., mask]
    den = np.sqrt((b * b).sum())
    return float(np.sqrt(((a - b) ** 2).sum()) / den) if den > 0 else float(np.abs(a).max())


def compare(gpu, ora, keys=("u", "v", "sigma")):
    return {k: rel_l2(gpu[k], ora[k], ora["mask"]) for k in keys}


def _table(dtype, cols):
    t = np.zeros(len(cols["node"]), dtype=dtype)
    for k in ("node", "dir", "bc", "bc2", "q", "n0", "n1"):
        t[k] = cols[k]
    return t


def run_gpu_tables(nt, cols, bcs, lam, steps, time_block=0, in_place=False, storage="f32"):
    """run_gpu for a node mask and cut-link columns given directly (not built
    from an analytic geometry)."""
    from paper_2208_04088_gb300 import _native as N
    from paper_2208_04088_gb300 import workloads as W
    d = N.Desc(nt, _table(N.LINK_DTYPE, cols), bcs, lam, W.MU, W.RHO0, tau=W.TAU,
               storage=storage, time_block=time_block, in_place=in_place)
    s = N.Solver(d)
    s.step(steps)
    s.sync()
    F = s.fields_host()
    F["info"] = s.info()
    F["mask"] = nt.astype(bool)
    s.close()
    return F


def run_oracle_tables(oracle_mod, nt, cols, bcs, lam, steps):
    """run_oracle for the same tables; every link takes the curved rules, which
    reduce to the lattice-conforming ones at q = 1/2."""
    from paper_2208_04088_gb300 import workloads as W
    links = _table(oracle_mod.LINK_DTYPE, cols)
    links["curved"] = 1
    o = oracle_mod.Oracle(nt, links, bcs, lam=lam, mu=W.MU, rho0=W.RHO0, tau=W.TAU)
    o.step(steps)
    F = o.fields()
    return {"u": F["u"], "v": F["v"], "sigma": F["sigma"], "mask": nt.astype(bool)}


def random_geometry(rng, nmin=2, nmax=90):
    """Seeded random box, hole or crack (geometry arguments of lbm_geom_build);
    boundary-condition indices 0..3."""
    nx, ny = int(rng.integers(nmin, nmax)), int(rng.integers(nmin, nmax))
    edge_bc = tuple(int(b) for b in rng.integers(0, 3, 4))
    kind = int(rng.integers(0, 3))
    hole = crack = None
    if kind == 1:
        # centres anywhere (on half-integers too, or off the box), radii from
        # below one spacing to beyond the box
        cx = float(rng.choice([rng.uniform(-5, nx + 5), rng.integers(0, nx) + 0.5]))
        cy = float(rng.choice([rng.uniform(-5, ny + 5), rng.integers(0, ny) + 0.5]))
        hole = (cx, cy, float(rng.uniform(0.3, 0.6 * max(nx, ny))), 3)
    elif kind == 2:
        ny += ny % 2
        length = int(rng.integers(1, nx + 3))
        x0 = int(rng.integers(0, nx)) if rng.random() < 0.5 else 0
        crack = (length, 3, x0)
    return dict(nx=nx, ny=ny, edge_bc=edge_bc, hole=hole, crack=crack)


# Rounding operations of FP32 arithmetic on the longest path from a stored
# population to the population stored one step later in the library's
# collision (raw moments 4, relaxation 4, inverse transform 2).
FP32_ROUNDINGS_PER_STEP = 10


def rounding_floor(oracle_mod, nt, links, bcs, lam, steps, seed=0, amp=2.0 ** -24):
    """The FP32 rounding floor of a problem, measured on the oracle: after
    every step each stored deviation f - f_rest is multiplied by 1 + e, e
    uniform in [-amp, amp] (one FP32 rounding, amp = 2^-24), and the fields at
    `steps` are compared with the clean run (relative L2 per field).  Errors of
    independent roundings add in quadrature, so a path of n roundings per step
    has a floor of about sqrt(n) times this."""
    from paper_2208_04088_gb300 import workloads as W
    import numpy as np
    mask = nt.astype(bool)
    clean = oracle_mod.Oracle(nt, links, bcs, lam=lam, mu=W.MU, rho0=W.RHO0, tau=W.TAU)
    clean.step(steps)
    A = clean.fields()
    clean.close()
    A["mask"] = mask
    o = oracle_mod.Oracle(nt, links, bcs, lam=lam, mu=W.MU, rho0=W.RHO0, tau=W.TAU)
    rng = np.random.default_rng(seed)
    rest = np.zeros((nt.shape[0], nt.shape[1], 9))
    rest[mask] = oracle_mod.feq(W.RHO0, (0.0, 0.0), (0.0, 0.0, 0.0))
    for _ in range(steps):
        o.step(1)
        f, u = o.state()
        d = f - rest
        d *= 1.0 + amp * rng.uniform(-1.0, 1.0, d.shape)
        o.set_state(rest + d, u, o.t)
    B = o.fields()
    o.close()
    return compare(B, A)
