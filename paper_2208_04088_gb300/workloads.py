"""Seeded synthetic workloads shaped like the paper's benchmark problems.

This module only states problem parameters (lattice size, material ratio,
geometry, boundary data, step counts); it holds none of the method's
arithmetic.  Both the CUDA library and the FP64 oracle consume what it
returns, so it is the one module the two sides share.

Boundary-condition kinds and profiles use the integer codes of the C ABI
(``include/lbm.h``):
  kind 0 Dirichlet (value = d(u*)/dt), 1 traction (value = t*),
       2 pressure (value[0] = p, t* = -p n), 3 stress (value = xx, yy, xy; t* = sigma n)
  profile 0 Heaviside step at t = 0, 1 linear ramp over t_ramp steps then hold.

Edge order for ``edge_bc`` is (left, right, bottom, top).
Everything is in lattice units: dx = dt = 1, rho0 = 1, mu = 1/3 (the isotropy
condition of Sec. 5.1 fixes c_s^2 = mu/rho0 = 1/3).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

DIRICHLET, TRACTION, PRESSURE, STRESS = 0, 1, 2, 3
STEP, RAMP = 0, 1

MU = 1.0 / 3.0
RHO0 = 1.0
TAU = 0.55  # tau_bar / dt, Sec. 3 and Sec. 5


@dataclasses.dataclass
class Workload:
    name: str
    nx: int
    ny: int
    steps: int
    lam_over_mu: float = 1.0  # 1.0 is the Poisson solid, nu = 1/4
    edge_bc: Tuple[int, int, int, int] = (0, 0, 0, 0)
    hole: Optional[Tuple[float, float, float, int]] = None  # (cx, cy, R, bc)
    crack: Optional[Tuple[int, ...]] = None  # (length, bc[, first column]); edge crack if 0
    bcs: List[dict] = dataclasses.field(default_factory=list)
    tau: float = TAU
    # Neumann wall values at the boundary node instead of the extrapolation of
    # Sec. 4 (an option of the library and the oracle, off = the paper's rule)
    wall_node: bool = False

    @property
    def lam(self) -> float:
        return self.lam_over_mu * MU

    @property
    def mu(self) -> float:
        return MU

    @property
    def rho0(self) -> float:
        return RHO0

    @property
    def nu(self) -> float:
        """Poisson's ratio of the plane-strain solid, lambda / (2 (lambda + mu))."""
        return self.lam / (2.0 * (self.lam + self.mu))

    @property
    def cd(self) -> float:
        """Dilatational wave speed sqrt((lambda + 2 mu)/rho0), lattice units."""
        return math.sqrt((self.lam + 2.0 * self.mu) / self.rho0)

    @property
    def nodes(self) -> int:
        return self.nx * self.ny

    def geometry_args(self) -> dict:
        return dict(nx=self.nx, ny=self.ny, edge_bc=self.edge_bc, hole=self.hole,
                    crack=self.crack)


def bc(kind, value, profile=STEP, t_ramp=0.0) -> dict:
    v = list(value) + [0.0] * (3 - len(value))
    return dict(kind=int(kind), value=tuple(float(a) for a in v), profile=int(profile),
                t_ramp=float(t_ramp))


def square_plate(n: int = 64, steps: int = 500, load: float = 1e-3,
                 lam_over_mu: float = 1.0) -> Workload:
    """Plain method check: left edge clamped (u* = 0), right edge a Heaviside
    traction sigma_xx = load, top and bottom traction-free, all lattice-conforming."""
    return Workload(
        name=f"square_plate_{n}x{n}", nx=n, ny=n, steps=steps, lam_over_mu=lam_over_mu,
        edge_bc=(0, 1, 2, 2),
        bcs=[bc(DIRICHLET, (0.0, 0.0)), bc(TRACTION, (load, 0.0)), bc(TRACTION, (0.0, 0.0))])


def hole_plate(nx: int = 1024, ny: int = 512, radius: float = 64.0, steps: int = 20000,
               load: float = 1e-3, lam_over_mu: float = 1.0, profile: int = STEP,
               t_ramp: float = 0.0) -> Workload:
    """Plate with a centred circular hole (curved, traction-free) under a
    Heaviside tension traction t* = load * n on the left and right edges;
    top, bottom and hole traction-free (Sec. 5.1 geometry, tension axis x)."""
    cx, cy = 0.5 * (nx - 1), 0.5 * (ny - 1)
    return Workload(
        name=f"hole_plate_{nx}x{ny}_R{radius:g}", nx=nx, ny=ny, steps=steps,
        lam_over_mu=lam_over_mu, edge_bc=(0, 0, 1, 1), hole=(cx, cy, float(radius), 1),
        bcs=[bc(PRESSURE, (-load,), profile, t_ramp), bc(TRACTION, (0.0, 0.0))])


def edge_crack(n: int = 2048, length: int = 512, steps: int = 1500, sigma0: float = 1e-3,
               lam_over_mu: float = 1.0, ny: Optional[int] = None) -> Workload:
    """Suddenly loaded stationary crack: an edge crack of the given length from
    the left edge on y = ny/2 - 1/2, both faces under a step pressure sigma0,
    all outer edges traction-free (Sec. 5.2)."""
    ny = n if ny is None else ny
    return Workload(
        name=f"edge_crack_{n}x{ny}_L{length}", nx=n, ny=ny, steps=steps,
        lam_over_mu=lam_over_mu, edge_bc=(0, 0, 0, 0), crack=(int(length), 1),
        bcs=[bc(TRACTION, (0.0, 0.0)), bc(PRESSURE, (sigma0,))])


def centre_crack(length: int = 100, steps: int = 210, sigma0: float = 1e-3,
                 lam_over_mu: float = 1.0, side: Optional[int] = None) -> Workload:
    """The centre crack of Sec. 5.2: a crack of the given length in the middle
    of a square plate of side 4 x length (the paper: 400 x 400 nodes, crack
    length 100), faces under a step pressure sigma0, outer edges traction-free."""
    side = 4 * length if side is None else side
    x0 = (side - length) // 2
    return Workload(
        name=f"centre_crack_{side}x{side}_L{length}", nx=side, ny=side, steps=steps,
        lam_over_mu=lam_over_mu, edge_bc=(0, 0, 0, 0), crack=(int(length), 1, int(x0)),
        bcs=[bc(TRACTION, (0.0, 0.0)), bc(PRESSURE, (sigma0,))])


# Material of the paper's crack run: c_s^2 / c_d^2 = 0.3611 (nu = 0.2174).
CRACK_PAPER_LAM_OVER_MU = 1.0 / 0.3611 - 2.0
# Non-Poisson plate of Sec. 5.1: c_d^2 / c_s^2 = 2.8 (nu = 2/9).
PLATE_NONPOISSON_LAM_OVER_MU = 0.8

# The five benchmark configurations (sizes and step counts as specified).
CONFIG1 = square_plate(64, 500)
CONFIG2 = hole_plate(1024, 512, 64.0, 20000)
CONFIG2_DOWNSCALE = hole_plate(256, 128, 16.0, 5000)
CONFIG3 = edge_crack(2048, 512, 1500)


def batched_instances(count: int = 256, seed: int = 4, steps: int = 5000) -> List[Workload]:
    """Seeded plate-with-hole instances: side a uniform in {128, 256, 512, 1024},
    aspect 1:1 or 2:1 (nx = a, ny = a or a/2), radius uniform in 8..min/8,
    traction amplitude uniform in [1e-4, 1e-3]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        a = int(rng.choice([128, 256, 512, 1024]))
        ny = a if rng.integers(0, 2) == 0 else a // 2
        r = int(rng.integers(8, min(a, ny) // 8 + 1))
        load = float(rng.uniform(1e-4, 1e-3))
        out.append(hole_plate(a, ny, float(r), steps, load))
    return out


def serving_trace(count: int = 500, seed: int = 5, rate: float = 50.0,
                  min_side: int = 64, max_side: int = 2048,
                  min_steps: int = 1000, max_steps: int = 50000):
    """Seeded request trace: Poisson arrivals at `rate` per second; geometry
    uniform over {square plate, hole plate, crack}; side log-uniform over the
    powers of two in [min_side, max_side]; steps log-uniform in
    [min_steps, max_steps]; load amplitude uniform in [1e-4, 1e-3].
    Returns a list of (arrival_time_s, Workload)."""
    rng = np.random.default_rng(seed)
    sides = [2 ** k for k in range(int(math.log2(min_side)), int(math.log2(max_side)) + 1)]
    t = 0.0
    out = []
    for _ in range(count):
        t += float(rng.exponential(1.0 / rate))
        kind = int(rng.integers(0, 3))
        side = int(rng.choice(sides))
        steps = int(round(math.exp(rng.uniform(math.log(min_steps), math.log(max_steps)))))
        load = float(rng.uniform(1e-4, 1e-3))
        if kind == 0:
            w = square_plate(side, steps, load)
        elif kind == 1:
            w = hole_plate(side, side, float(max(4, side // 8)), steps, load)
        else:
            w = edge_crack(side, max(2, side // 4), steps, load)
        out.append((t, w))
    return out


# Direction numbering of the link tables (the C ABI's lbm_link.dir): 1 +x,
# 2 +y, 3 -x, 4 -y, 5 (+,+), 6 (-,+), 7 (-,-), 8 (+,-).
_DIRS = ((0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1))
_OPPOSITE = (0, 3, 4, 1, 2, 7, 8, 5, 6)


def fragmented_solid(nx: int, ny: int, seed: int, void_frac: float = 0.2,
                     crack_frac: float = 0.05, nbcs: int = 4):
    """Seeded node mask and cut-link table of a fragmented solid, a stress case
    for the boundary rules (no geometry of the paper has one).

    Each node is void with probability `void_frac`.  Every link from a material
    node to a void node or out of the box is cut; each link between two
    material nodes is cut with probability `crack_frac`, on both sides (a crack
    through the link).  A cut's wall distance q is 1/2 with probability 1/4 and
    otherwise uniform in (0, 1]; across a crack the far side gets 1 - q (drawn
    in (0, 1) there) and the opposite normal.  Normals are uniform unit vectors;
    boundary-condition indices are uniform in range(nbcs); no corner links.

    Returns node_type (uint8, ny x nx) and a dict of equal-length columns
    node, dir, bc, bc2, q, n0, n1 in (node, dir) order.
    """
    rng = np.random.default_rng(seed)
    mat = (rng.random((ny, nx)) >= void_frac).astype(np.uint8)
    crack = rng.random((ny, nx, 9)) < crack_frac
    u = rng.random((ny, nx, 9))
    q = np.where(rng.random((ny, nx, 9)) < 0.25, 0.5, 1.0 - u)  # 1 - u is in (0, 1]
    q_crack = np.clip(u, 1e-3, 1.0 - 1e-3)
    ang = rng.uniform(0.0, 2.0 * math.pi, (ny, nx, 9))
    bcs = rng.integers(0, nbcs, (ny, nx, 9))
    cut = {}
    for y in range(ny):
        for x in range(nx):
            if not mat[y, x]:
                continue
            for i in range(1, 9):
                tx, ty = x + _DIRS[i][0], y + _DIRS[i][1]
                inside = 0 <= tx < nx and 0 <= ty < ny
                if not inside or not mat[ty, tx]:
                    cut[(y * nx + x, i)] = (int(bcs[y, x, i]), float(q[y, x, i]),
                                            math.cos(ang[y, x, i]), math.sin(ang[y, x, i]))
                elif (ty * nx + tx) > (y * nx + x) and crack[y, x, i]:
                    # one draw per material-material link, taken at its lower node
                    qa = float(q_crack[y, x, i])
                    c, s = math.cos(ang[y, x, i]), math.sin(ang[y, x, i])
                    b = int(bcs[y, x, i])
                    cut[(y * nx + x, i)] = (b, qa, c, s)
                    cut[(ty * nx + tx, _OPPOSITE[i])] = (b, 1.0 - qa, -c, -s)
    keys = sorted(cut)
    cols = {
        "node": np.array([k[0] for k in keys], dtype=np.int32),
        "dir": np.array([k[1] for k in keys], dtype=np.int32),
        "bc": np.array([cut[k][0] for k in keys], dtype=np.int32),
        "bc2": np.full(len(keys), -1, dtype=np.int32),
        "q": np.array([cut[k][1] for k in keys], dtype=np.float64),
        "n0": np.array([cut[k][2] for k in keys], dtype=np.float64),
        "n1": np.array([cut[k][3] for k in keys], dtype=np.float64),
    }
    return mat, cols


def fragmented_bcs(load: float = 5e-4) -> List[dict]:
    """The four boundary conditions `fragmented_solid` indexes: a moving wall
    (ramped), a traction, a pressure (ramped) and a general stress."""
    return [bc(DIRICHLET, (0.4 * load, -0.3 * load), RAMP, 20.0),
            bc(TRACTION, (0.6 * load, 0.2 * load)),
            bc(PRESSURE, (0.5 * load,), RAMP, 10.0),
            bc(STRESS, (0.7 * load, -0.4 * load, 0.3 * load))]
