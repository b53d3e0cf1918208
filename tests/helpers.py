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
