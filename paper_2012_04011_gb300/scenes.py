"""Seeded synthetic inputs: grids, obstacle scenes and the initial value V0.

This module builds inputs only.  It holds none of the numerical scheme: no
differences, Hamiltonian, dissipation, time step or BRT min.  Both the CUDA
path and the FP64 oracle consume the V0 arrays it produces, so the two sides
always start from the same bytes.

V0 follows Sec. IV-A, Eq. (init_V): the signed xy-distance to a round
obstacle, sqrt((x - x_o)^2 + (y - y_o)^2) - R, replicated over v and theta.
Several obstacles combine by a pointwise min (the union of the target sets
{V0 <= 0}).  Axis-aligned rectangles (used by the 128x128x64x96 workload, not
in the paper) use the exact rectangle signed distance.

Workloads (the paper's lab scenes are not published, so seeded random
obstacles stand in for them; Sec. IV-A, Fig. 4):
  car4d_31x31x11x16   6 circles, T = 1.0 s
  car4d_60x60x20x36   12 circles, T = 2.0 s (the paper's grid size)
  car4d_128x128x64x96 28 circles + 4 rectangles, T = 2.0 s
  batch64             64 instances, uneven grids, 4-16 circles, T = 1.5 s
Domain for all: x, y in [-5, 5], v in [0, 4], theta in [-pi, pi) periodic;
a_max = 1.5, w_max = 1.0, CFL 0.8.  Circles: centres uniform in [-4, 4]^2,
radii uniform in [0.3, 1.0].  Rectangles: centres uniform in [-4, 4]^2,
half-sizes uniform in [0.2, 1.0].

The paper's own experiment (Sec. IV-A) is paper_room(): the 6 m x 4 m room
on 60x60x20x36 points at 0.1 m, 0.067 m, 0.2 m/s and 2 pi/36 rad, the
steering car (a in [-1.5, 1.5], delta in [-pi/18, pi/18], L = 0.3 m), cones
inflated to R = 0.75 m, horizon 0.5 s in steps of the reported 0.007497 s
(67 steps).  The cone placements are not published: seeded positions in the
room stand in for its three environments.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2012040110

DOMAIN_LO = (-5.0, -5.0, 0.0, -math.pi)
DOMAIN_HI = (5.0, 5.0, 4.0, math.pi)
PERIODIC_THETA = 0b1000  # bit 3: theta wraps
A_MAX = 1.5
W_MAX = 1.0
CFL = 0.8


@dataclass
class GridSpec:
    """Points per axis (x, y, v, theta) and the axis bounds."""
    n: tuple
    lo: tuple = DOMAIN_LO
    hi: tuple = DOMAIN_HI
    periodic: int = PERIODIC_THETA

    @property
    def ncell(self) -> int:
        return int(np.prod(self.n))

    def axis(self, d: int) -> np.ndarray:
        """Grid states on axis d: lo + i*h, h = (hi-lo)/(N-1), or (hi-lo)/N if periodic."""
        N = self.n[d]
        h = (self.hi[d] - self.lo[d]) / (N if (self.periodic >> d) & 1 else N - 1)
        return self.lo[d] + np.arange(N, dtype=np.float64) * h


@dataclass
class Scene:
    """Obstacles: circles (x_o, y_o, R) and axis-aligned rectangles (cx, cy, hx, hy)."""
    circles: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    rects: np.ndarray = field(default_factory=lambda: np.zeros((0, 4)))

    def copy(self) -> "Scene":
        return Scene(self.circles.copy(), self.rects.copy())


@dataclass
class Workload:
    name: str
    grid: GridSpec
    scene: Scene
    T: float
    seed: int
    a_max: float = A_MAX
    w_max: float = W_MAX
    cfl: float = CFL


def random_scene(rng: np.random.Generator, n_circles: int, n_rects: int = 0) -> Scene:
    c = np.empty((n_circles, 3))
    c[:, 0:2] = rng.uniform(-4.0, 4.0, size=(n_circles, 2))
    c[:, 2] = rng.uniform(0.3, 1.0, size=n_circles)
    r = np.empty((n_rects, 4))
    r[:, 0:2] = rng.uniform(-4.0, 4.0, size=(n_rects, 2))
    r[:, 2:4] = rng.uniform(0.2, 1.0, size=(n_rects, 2))
    return Scene(c, r)


def signed_distance_xy(grid: GridSpec, scene: Scene) -> np.ndarray:
    """min over obstacles of the signed xy-distance on the (N1, N2) plane."""
    x = grid.axis(0)[:, None]
    y = grid.axis(1)[None, :]
    sd = np.full((grid.n[0], grid.n[1]), np.inf)
    for xo, yo, R in scene.circles:
        sd = np.minimum(sd, np.sqrt((x - xo) ** 2 + (y - yo) ** 2) - R)
    for cx, cy, hx, hy in scene.rects:
        qx = np.abs(x - cx) - hx
        qy = np.abs(y - cy) - hy
        outside = np.sqrt(np.maximum(qx, 0.0) ** 2 + np.maximum(qy, 0.0) ** 2)
        inside = np.minimum(np.maximum(qx, qy), 0.0)
        sd = np.minimum(sd, outside + inside)
    if not np.all(np.isfinite(sd)):
        raise ValueError("scene has no obstacles")
    return sd


def initial_value(grid: GridSpec, scene: Scene) -> np.ndarray:
    """V0[i, j, k, l] (FP64, C order, theta fastest) from Eq. (init_V)."""
    sd = signed_distance_xy(grid, scene)
    v0 = np.broadcast_to(sd[:, :, None, None], grid.n)
    return np.ascontiguousarray(v0, dtype=np.float64)


def _single(name: str, n, n_circles: int, n_rects: int, T: float, seed: int) -> Workload:
    rng = np.random.default_rng(seed)
    return Workload(name, GridSpec(tuple(n)), random_scene(rng, n_circles, n_rects), T, seed)


def workload(name: str) -> Workload:
    """The named single-instance workloads."""
    if name == "car4d_31x31x11x16":
        return _single(name, (31, 31, 11, 16), 6, 0, 1.0, SEED_BASE + 0)
    if name == "car4d_60x60x20x36":
        return _single(name, (60, 60, 20, 36), 12, 0, 2.0, SEED_BASE + 1)
    if name == "car4d_128x128x64x96":
        return _single(name, (128, 128, 64, 96), 28, 4, 2.0, SEED_BASE + 3)
    raise KeyError(name)


WORKLOADS = ("car4d_31x31x11x16", "car4d_60x60x20x36", "car4d_128x128x64x96")


def batch_workloads(count: int = 64, seed: int = SEED_BASE + 2):
    """Independent instances with uneven grids: N1, N2 in {40, 50, 60}, N3 in
    [16, 24], N4 in [24, 36], 4-16 circles each, T = 1.5 s."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        n = (int(rng.choice([40, 50, 60])), int(rng.choice([40, 50, 60])),
             int(rng.integers(16, 25)), int(rng.integers(24, 37)))
        sc = random_scene(rng, int(rng.integers(4, 17)))
        out.append(Workload(f"batch{b}", GridSpec(n), sc, 1.5, seed))
    return out


def custom_workload(n, n_circles: int = 4, n_rects: int = 0, T: float = 0.5, seed: int = SEED_BASE + 99,
                    a_max: float = A_MAX, w_max: float = W_MAX, cfl: float = CFL) -> Workload:
    """Seeded scene on an arbitrary grid (tests use it for ragged and tiny shapes)."""
    rng = np.random.default_rng(seed)
    return Workload(f"custom{tuple(n)}", GridSpec(tuple(int(x) for x in n)), random_scene(rng, n_circles, n_rects),
                    T, seed, a_max, w_max, cfl)


# ---------------------------------------------------------------- the paper's room

PAPER_ROOM_N = (60, 60, 20, 36)
PAPER_ROOM_LO = (0.0, 0.0, 0.0, -math.pi)
PAPER_ROOM_HI = (59 * 0.1, 59 * 0.067, 19 * 0.2, math.pi)  # x 6 m, y 4 m, v up to 3.8 m/s
PAPER_STEER = (1.5, math.pi / 18, 0.3)                        # a_max, delta_max, L
PAPER_CONE_R = 0.75
PAPER_T = 0.5
PAPER_DT = 0.007497  # the largest stable step the paper reports for its grid


def paper_room_cfl(grid: GridSpec, steer=PAPER_STEER, dt: float = PAPER_DT) -> float:
    """Courant number at which the CFL step of the grid is dt: the step is
    CFL / sum_d alpha_d^max / dx_d with alpha^max = (v_max, v_max, a_max,
    v_max tan(delta_max) / L) (cos and sin reach 1 on this theta grid)."""
    h = [(grid.hi[d] - grid.lo[d]) / (grid.n[d] if (grid.periodic >> d) & 1 else grid.n[d] - 1) for d in range(4)]
    vmax = max(abs(grid.lo[2]), abs(grid.hi[2]))
    a_max, d_max, L = steer
    s = vmax / h[0] + vmax / h[1] + a_max / h[2] + vmax * math.tan(d_max) / L / h[3]
    return dt * s


def paper_room(env: int = 1, n_cones: int = 3) -> Workload:
    """The room of Sec. IV-A with n_cones seeded cones (env selects the
    seed; the paper's three environments are not published)."""
    rng = np.random.default_rng(SEED_BASE + 10 + env)
    cones = np.empty((n_cones, 3))
    cones[:, 0] = rng.uniform(0.8, PAPER_ROOM_HI[0] - 0.8, n_cones)
    cones[:, 1] = rng.uniform(0.8, PAPER_ROOM_HI[1] - 0.8, n_cones)
    cones[:, 2] = PAPER_CONE_R
    grid = GridSpec(PAPER_ROOM_N, PAPER_ROOM_LO, PAPER_ROOM_HI)
    return Workload(f"paper_room_env{env}", grid, Scene(cones), PAPER_T, SEED_BASE + 10 + env,
                    a_max=PAPER_STEER[0], w_max=0.0, cfl=paper_room_cfl(grid))


# ---------------------------------------------------------------- serving trace

SERVING_SIZES = ((31, 31, 11, 16), (60, 60, 20, 36), (80, 80, 25, 40), (100, 100, 30, 48))
SERVING_T = 0.5  # the paper's horizon (Sec. IV-A)


@dataclass
class Request:
    """One re-solve request: arrival time (s), grid and the scene at that time."""
    t_arrival: float
    workload: Workload

    def v0_xy(self) -> np.ndarray:
        return signed_distance_xy(self.workload.grid, self.workload.scene)


def perturb_scene(rng: np.random.Generator, scene: Scene, max_circles: int = 16) -> Scene:
    """1-4 changes: shift an obstacle by up to 0.5 m, or add a circle of
    radius 0.3-1.0 m (the oldest circle is dropped beyond max_circles)."""
    s = scene.copy()
    for _ in range(int(rng.integers(1, 5))):
        if rng.random() < 0.5 and len(s.circles) > 0:
            i = int(rng.integers(0, len(s.circles)))
            ang, r = rng.uniform(0, 2 * np.pi), rng.uniform(0.0, 0.5)
            s.circles[i, 0:2] = np.clip(s.circles[i, 0:2] + r * np.array([np.cos(ang), np.sin(ang)]), -4.5, 4.5)
        else:
            c = np.array([[*rng.uniform(-4.0, 4.0, size=2), rng.uniform(0.3, 1.0)]])
            s.circles = np.concatenate([s.circles, c])[-max_circles:]
    return s


def serving_trace(rate_hz: float, duration_s: float, seed: int = SEED_BASE + 4, sizes=SERVING_SIZES,
                  T: float = SERVING_T):
    """Poisson arrivals at rate_hz for duration_s seconds; each request
    perturbs the resident scene and asks for a re-solve on a grid drawn from
    sizes."""
    rng = np.random.default_rng(seed)
    scene = random_scene(rng, 8)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t > duration_s:
            break
        scene = perturb_scene(rng, scene)
        n = sizes[int(rng.integers(0, len(sizes)))]
        out.append(Request(t, Workload(f"req{len(out)}", GridSpec(tuple(n)), scene.copy(), T, seed)))
    return out
