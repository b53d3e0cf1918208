"""Host-side checks of the C ABI (no GPU needed).

* liblbm.so loads and exports every function include/lbm.h declares.
* The library's geometry builder (its own code) produces node masks and
  cut-link tables bit-identical to the oracle's independent classifier.
* Descriptor validation rejects inconsistent tables with LBM_ERR_ARG.
"""
import os
import re

import numpy as np
import pytest

from helpers import random_geometry

from paper_2208_04088_gb300 import _native as N
from paper_2208_04088_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = N.load()
    declared = _declared_functions()
    assert len(declared) >= 12
    for name in declared:
        assert hasattr(lib, name), name
        assert name in N.SIGNATURES, name


@pytest.mark.parametrize("wl", [W.square_plate(64, 0), W.hole_plate(256, 128, 16.0, 0),
                                W.hole_plate(1024, 512, 64.0, 0), W.hole_plate(101, 77, 12.5, 0),
                                W.edge_crack(128, 40, 0), W.edge_crack(64, 64, 0, ny=32),
                                W.centre_crack(25, 0), W.centre_crack(100, 0)],
                         ids=lambda w: w.name)
def test_geometry_tables_bit_exact_with_oracle(oracle_mod, wl):
    nt_o, lk_o = oracle_mod.geometry(**wl.geometry_args())
    nt_l, lk_l = N.lbm_geom_build(**wl.geometry_args())
    assert np.array_equal(nt_o, nt_l)
    assert len(lk_o) == len(lk_l)
    for f in ("node", "dir", "bc", "bc2"):
        assert np.array_equal(lk_o[f], lk_l[f]), f
    for f in ("q", "n0", "n1"):
        assert np.array_equal(lk_o[f].view(np.uint64), lk_l[f].view(np.uint64)), f


def _desc(wl, **kw):
    return N.desc_from_workload(wl, **kw)


def test_workspace_size_accounts_for_storage():
    wl = W.hole_plate(256, 128, 16.0, 0)
    b32 = N.lbm_workspace_size(_desc(wl, storage="f32"))
    b16 = N.lbm_workspace_size(_desc(wl, storage="f16"))
    plane = 256 * 128
    # two buffers with 2 bytes less per value, and the displacement record:
    # (u, compensation) float4 with FP32 storage, (u_x, u_y) float2 with 16-bit
    assert b32 - b16 >= 2 * 9 * plane * 2 + 8 * plane
    assert b32 > 2 * 9 * plane * 4 + 16 * plane
    assert b16 > 2 * 9 * plane * 2 + 8 * plane


def test_validation_rejects_bad_tables():
    wl = W.square_plate(16, 0)
    nt, links = N.lbm_geom_build(**wl.geometry_args())
    # a missing cut link leaves a node linked to the outside
    d = N.Desc(nt, links[1:], wl.bcs, wl.lam, wl.mu)
    with pytest.raises(N.LbmError) as e:
        N.lbm_workspace_size(d)
    assert e.value.status == N.LBM_ERR_ARG
    # duplicate link
    d = N.Desc(nt, np.concatenate([links, links[:1]]), wl.bcs, wl.lam, wl.mu)
    with pytest.raises(N.LbmError):
        N.lbm_workspace_size(d)
    # bad wall distance
    bad = links.copy()
    bad["q"][0] = 0.0
    with pytest.raises(N.LbmError):
        N.lbm_workspace_size(N.Desc(nt, bad, wl.bcs, wl.lam, wl.mu))
    # isotropy condition dx/(sqrt(3) dt) = sqrt(mu/rho0) violated
    with pytest.raises(N.LbmError):
        N.lbm_workspace_size(N.Desc(nt, links, wl.bcs, wl.lam, wl.mu, dx=1.0, dt=0.5))
    # tau must exceed 1/2
    with pytest.raises(N.LbmError):
        N.lbm_workspace_size(N.Desc(nt, links, wl.bcs, wl.lam, wl.mu, tau=0.5))
    # out-of-range bc index
    bad = links.copy()
    bad["bc"][0] = 99
    with pytest.raises(N.LbmError):
        N.lbm_workspace_size(N.Desc(nt, bad, wl.bcs, wl.lam, wl.mu))
    assert "bad cut link" in N.lbm_last_error()


def test_physical_units_are_accepted():
    # the plate of Sec. 5.1 in its own units: l = 1, dx = 0.0125 l, mu = 1, rho = 1,
    # c_s = 1, dt = dx/(sqrt(3) c_s)
    wl = W.square_plate(80, 0)
    nt, links = N.lbm_geom_build(**wl.geometry_args())
    dx = 0.0125
    d = N.Desc(nt, links, wl.bcs, lam=1.0, mu=1.0, rho0=1.0, dx=dx, dt=dx / np.sqrt(3.0))
    assert N.lbm_workspace_size(d) > 0
    # the paper's printed, rounded time step 7.217e-3 l/c_s is within the tolerance
    d = N.Desc(nt, links, wl.bcs, lam=1.0, mu=1.0, rho0=1.0, dx=dx, dt=7.217e-3)
    assert N.lbm_workspace_size(d) > 0


def test_time_block_selection_and_validation():
    """lbm_desc.time_block: 0 (default: blocked where faster), 1 (one step per launch) or
    LBM_TIME_BLOCK (temporal blocking, FP32 storage, nx >= 128);
    the blocked form adds the 8-byte node words and its block table to the
    workspace."""
    wl = W.hole_plate(256, 128, 16.0, 0)
    plane = 256 * 128
    one = N.lbm_workspace_size(_desc(wl, time_block=1))
    blk = N.lbm_workspace_size(_desc(wl, time_block=N.LBM_TIME_BLOCK))
    dflt = N.lbm_workspace_size(_desc(wl))
    # node words (8 bytes per node) and the block table (16 bytes per block and
    # 8 for its measured cycles; at most max(strips, 4096) + strips blocks of
    # 112-column strips)
    strips = (256 + 111) // 112
    table = (max(strips, 4096) + strips) * 24
    assert blk - one == (8 * plane + 255) // 256 * 256 + (table + 255) // 256 * 256
    # the default is blocked only where that is the faster form: at least 2^21
    # nodes, lambda = mu and at most one boundary node off box edges and crack
    # faces per 800 nodes
    assert dflt == one
    crack = W.edge_crack(2048, 512, 0)
    assert N.lbm_workspace_size(_desc(crack)) == \
        N.lbm_workspace_size(_desc(crack, time_block=N.LBM_TIME_BLOCK))
    # a hole of radius 512 in a 2048^2 plate: about one curved-wall node per
    # 1022 nodes, blocked; radius 900 (one per 582): one step per launch
    hole = W.hole_plate(2048, 2048, 512.0, 0)
    assert N.lbm_workspace_size(_desc(hole)) == \
        N.lbm_workspace_size(_desc(hole, time_block=N.LBM_TIME_BLOCK))
    big_hole = W.hole_plate(2048, 2048, 900.0, 0)
    assert N.lbm_workspace_size(_desc(big_hole)) == \
        N.lbm_workspace_size(_desc(big_hole, time_block=1))
    # the default falls back to one step per launch where blocking is unsupported
    assert N.lbm_workspace_size(_desc(wl, storage="f16")) == \
        N.lbm_workspace_size(_desc(wl, storage="f16", time_block=1))
    for bad in (2, 3, 16, -1):
        with pytest.raises(N.LbmError, match="LBM_ERR_ARG"):
            N.lbm_workspace_size(_desc(wl, time_block=bad))
    with pytest.raises(N.LbmError, match="LBM_ERR_ARG"):
        N.lbm_workspace_size(_desc(wl, storage="bf16", time_block=N.LBM_TIME_BLOCK))
    # lambda != mu is blocked too (4 steps per launch): the same extra tables
    nonpoisson = W.hole_plate(256, 128, 16.0, 0, lam_over_mu=0.8)
    assert N.lbm_workspace_size(_desc(nonpoisson, time_block=N.LBM_TIME_BLOCK)) - \
        N.lbm_workspace_size(_desc(nonpoisson, time_block=1)) == blk - one
    # ... but its default is one step per launch (the faster form there)
    assert N.lbm_workspace_size(_desc(nonpoisson)) == \
        N.lbm_workspace_size(_desc(nonpoisson, time_block=1))
    narrow = W.square_plate(64, 0)
    with pytest.raises(N.LbmError, match="LBM_ERR_ARG"):
        N.lbm_workspace_size(_desc(narrow, time_block=N.LBM_TIME_BLOCK))
    assert N.lbm_workspace_size(_desc(narrow)) == N.lbm_workspace_size(_desc(narrow, time_block=1))


def test_in_place_streaming_selection_and_validation():
    """lbm_desc.streaming = LBM_STREAM_IN_PLACE: one population buffer (9
    planes padded by a ring of one node) instead of two, one step per launch,
    lambda = mu only."""
    wl = W.hole_plate(256, 128, 16.0, 0)
    two = N.lbm_workspace_size(_desc(wl, time_block=1))
    one = N.lbm_workspace_size(N.desc_from_workload(wl, in_place=True))
    # one buffer fewer; the ring widens the pitch of every per-node array here
    # (256 -> 320 columns), so less than a whole buffer is saved at this size
    buf_two = 9 * 4 * 256 * 128
    assert two - one >= buf_two // 2
    # temporal blocking keeps two buffers
    with pytest.raises(N.LbmError, match="LBM_ERR_ARG"):
        N.lbm_workspace_size(N.desc_from_workload(wl, time_block=N.LBM_TIME_BLOCK, in_place=True))
    # the default form with in-place streaming is one step per launch (no node words)
    crack = W.edge_crack(2048, 512, 0)
    assert N.lbm_workspace_size(N.desc_from_workload(crack, in_place=True)) < \
        N.lbm_workspace_size(N.desc_from_workload(crack, time_block=1))
    # lambda != mu: the source's density gradient would read overwritten populations
    nonpoisson = W.hole_plate(256, 128, 16.0, 0, lam_over_mu=0.8)
    with pytest.raises(N.LbmError, match="LBM_ERR_ARG"):
        N.lbm_workspace_size(N.desc_from_workload(nonpoisson, in_place=True))
    bad = N.desc_from_workload(wl)
    bad.c.streaming = 7
    with pytest.raises(N.LbmError, match="LBM_ERR_ARG"):
        N.lbm_workspace_size(bad)


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structures have the sizes and field offsets of the
    C structures in include/lbm.h (compiled here with the host C compiler)."""
    import shutil
    import subprocess
    import ctypes as C
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = {"lbm_desc": N.lbm_desc, "lbm_info": N.lbm_info, "lbm_bc": N.lbm_bc,
               "lbm_geom": N.lbm_geom, "lbm_launch_shape": N.lbm_launch_shape,
               "lbm_batch_stats": N.lbm_batch_stats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "lbm.h"', "int main(void) {"]
    c_names = {"lam": "lambda"}  # Python keyword avoided in the binding
    for sname, cls in structs.items():
        lines.append(f'printf("{sname} %zu\\n", sizeof({sname}));')
        for fname, _ in cls._fields_:
            cname = c_names.get(fname, fname)
            lines.append(f'printf("{sname}.{fname} %zu\\n", offsetof({sname}, {cname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                         text=True).stdout.split("\n") if l)
    for sname, cls in structs.items():
        assert int(out[sname]) == C.sizeof(cls), sname
        for fname, _ in cls._fields_:
            assert int(out[f"{sname}.{fname}"]) == getattr(cls, fname).offset, (sname, fname)


def _zero_links():
    return np.zeros(0, dtype=N.LINK_DTYPE)


def test_lattice_size_limits_and_empty_material():
    bcs = [W.bc(W.DIRICHLET, (0.0, 0.0))]
    for nx, ny in ((1, 8), (8, 1), (65536, 2), (2, 65536)):
        with pytest.raises(N.LbmError) as e:
            N.lbm_workspace_size(N.Desc(np.zeros((ny, nx), np.uint8), _zero_links(), bcs, W.MU, W.MU))
        assert e.value.status == N.LBM_ERR_ARG
        assert "2..65535" in N.lbm_last_error()
    # the smallest lattice, and one with no material node at all, are accepted
    assert N.lbm_workspace_size(N.Desc(np.zeros((2, 2), np.uint8), _zero_links(), bcs, W.MU, W.MU)) > 0
    assert N.lbm_workspace_size(N.Desc(np.zeros((64, 256), np.uint8), _zero_links(), bcs, W.MU, W.MU,
                                       time_block=N.LBM_TIME_BLOCK)) > 0
    # a material node without its cut links is rejected
    with pytest.raises(N.LbmError):
        N.lbm_workspace_size(N.Desc(np.ones((4, 4), np.uint8), _zero_links(), bcs, W.MU, W.MU))


DIRS = ((0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1))


@pytest.mark.parametrize("args", [(150, 45, 7, 0.2, 0.05), (40, 30, 3, 0.6, 0.05), (33, 17, 1, 0.0, 0.3)])
def test_fragmented_solid_tables(oracle_mod, args):
    """The seeded fragmented solid: every link from a material node to a void
    node or out of the box is cut, every cut between two material nodes is
    paired with the reverse link (q and 1 - q, opposite normals), and both the
    library and the oracle accept the tables."""
    nx, ny, seed, vf, cf = args
    nt, cols = W.fragmented_solid(nx, ny, seed, void_frac=vf, crack_frac=cf, nbcs=2)
    cut = {(int(n), int(d)): k for k, (n, d) in enumerate(zip(cols["node"], cols["dir"]))}
    assert len(cut) == len(cols["node"])
    assert np.all((cols["q"] > 0) & (cols["q"] <= 1)) and np.all(cols["bc2"] == -1)
    assert np.allclose(cols["n0"] ** 2 + cols["n1"] ** 2, 1.0)
    cracks = 0
    for y in range(ny):
        for x in range(nx):
            for i in range(1, 9):
                key = (y * nx + x, i)
                tx, ty = x + DIRS[i][0], y + DIRS[i][1]
                if not nt[y, x]:
                    assert key not in cut
                    continue
                if not (0 <= tx < nx and 0 <= ty < ny) or not nt[ty, tx]:
                    assert key in cut
                elif key in cut:
                    back = cut[(ty * nx + tx, (i + 1) % 4 + 1 if i <= 4 else (i - 3) % 4 + 5)]
                    k = cut[key]
                    assert cols["q"][k] + cols["q"][back] == pytest.approx(1.0, abs=1e-12)
                    assert cols["n0"][k] == -cols["n0"][back] and cols["n1"][k] == -cols["n1"][back]
                    cracks += 1
    assert cracks > 0  # every case draws some cracks
    bcs = [W.bc(W.DIRICHLET, (1e-4, 0.0)), W.bc(W.DIRICHLET, (0.0, 1e-4))]
    links = np.zeros(len(cols["node"]), dtype=N.LINK_DTYPE)
    for k in ("node", "dir", "bc", "bc2", "q", "n0", "n1"):
        links[k] = cols[k]
    assert N.lbm_workspace_size(N.Desc(nt, links, bcs, W.MU, W.MU)) > 0
    olinks = np.zeros(len(cols["node"]), dtype=oracle_mod.LINK_DTYPE)
    for k in ("node", "dir", "bc", "bc2", "q", "n0", "n1"):
        olinks[k] = cols[k]
    olinks["curved"] = 1
    o = oracle_mod.Oracle(nt, olinks, bcs, lam=W.MU, mu=W.MU)
    o.step(2)
    assert np.all(np.isfinite(o.fields()["u"]))


@pytest.mark.parametrize("seed", range(6))
def test_random_geometry_tables_bit_exact_with_oracle(oracle_mod, seed):
    """lbm_geom_build and the oracle's geometry, written apart, on seeded random
    boxes, holes and cracks: identical masks and bit-identical link tables, or
    both reject the arguments."""
    rng = np.random.default_rng(1000 + seed)
    for _ in range(25):
        g = random_geometry(rng)
        try:
            nt_o, lk_o = oracle_mod.geometry(**g)
        except ValueError:
            with pytest.raises(N.LbmError):
                N.lbm_geom_build(**g)
            continue
        nt_l, lk_l = N.lbm_geom_build(**g)
        assert np.array_equal(nt_o, nt_l), g
        assert len(lk_o) == len(lk_l), g
        for f in ("node", "dir", "bc", "bc2"):
            assert np.array_equal(lk_o[f], lk_l[f]), (f, g)
        for f in ("q", "n0", "n1"):
            assert np.array_equal(lk_o[f].view(np.uint64), lk_l[f].view(np.uint64)), (f, g)


def test_hole_covering_the_box_leaves_no_material(oracle_mod):
    g = dict(nx=12, ny=9, edge_bc=(0, 0, 0, 0), hole=(5.5, 4.0, 50.0, 1), crack=None)
    nt_o, lk_o = oracle_mod.geometry(**g)
    nt_l, lk_l = N.lbm_geom_build(**g)
    assert nt_o.sum() == 0 and nt_l.sum() == 0 and len(lk_o) == 0 and len(lk_l) == 0
