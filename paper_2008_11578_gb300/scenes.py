"""Seeded synthetic scenes shaped like the paper's workloads.

This module only draws inputs.  It holds none of the ORCA arithmetic, so both
the FP64 oracle and the CUDA path consume exactly the same arrays.

The paper (Sec. 4) describes its workloads only in words: start and end
regions, random spawns, two-way and four-way crossings, a goal per agent, and
timings averaged over such test cases.  It publishes no dataset.  The five
scene families below stand in for those workloads.  Every draw comes from
``numpy.random.default_rng(seed)`` in the order written in each function.

Agent types: 0 = pedestrian, 1 = vehicle (the two agent kinds of Sec. 3.1).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

PEDESTRIAN = 0
VEHICLE = 1


@dataclasses.dataclass
class OrcaParams:
    """Global ORCA parameters (Sec. 3 and 3.1).

    ``f[a][b]`` is the responsibility factor f_{A|B} that an agent of type
    ``a`` takes when avoiding an agent of type ``b`` (Sec. 3.1).  The default
    is the table of the paper's experiments (Sec. 4): f_{person|car} = 1,
    f_{car|person} = 0, and 1/2 for like pairs.
    """

    neighbor_dist: float = 10.0
    max_neighbors: int = 10
    time_horizon: float = 5.0
    dt: float = 0.25
    f: tuple = ((0.5, 1.0), (0.0, 0.5))
    # uniform grid over the scene box; cell width and height are tuning knobs
    # that never change results (the neighbour search is exact); height 0
    # means square cells
    cell_size: float = 2.0
    cell_height: float = 0.0
    origin: tuple = (0.0, 0.0)
    extent: tuple = (50.0, 50.0)
    # kinematic limits of vehicles (rad/s, m/s^2); 0 = off.  The paper's
    # proposed extension for vehicles (Sec. 5): extra linear constraints
    vehicle_turn_rate: float = 0.0
    vehicle_accel: float = 0.0

    def cell_dims(self, cell_size: float | None = None,
                  cell_height: float | None = None) -> tuple[float, float]:
        """(width, height) of a grid cell; a height of 0 or None means the
        width (square cells) unless the params fix a height."""
        w = float(self.cell_size if cell_size is None else cell_size)
        h = float(self.cell_height if cell_height is None else cell_height)
        if cell_size is not None and cell_height is None:
            h = 0.0
        return w, (h if h > 0.0 else w)

    def grid_dims(self, cell_size: float | None = None,
                  cell_height: float | None = None) -> tuple[int, int]:
        w, h = self.cell_dims(cell_size, cell_height)
        nx = max(1, int(math.ceil(self.extent[0] / w)))
        ny = max(1, int(math.ceil(self.extent[1] / h)))
        return nx, ny

    def f_array(self) -> np.ndarray:
        return np.asarray(self.f, dtype=np.float32).reshape(2, 2)


@dataclasses.dataclass
class Scene:
    """Structure-of-arrays agent state, all in original agent order."""

    pos: np.ndarray            # (N, 2) float32
    vel: np.ndarray            # (N, 2) float32
    goal: np.ndarray           # (N, 2) float32
    radius: np.ndarray         # (N,) float32
    max_speed: np.ndarray      # (N,) float32
    type: np.ndarray           # (N,) uint8
    params: OrcaParams
    route: np.ndarray | None = None       # (N,) int32, -1 = follow goal
    waypoints: np.ndarray | None = None   # (R, W, 2) float32
    wp_idx: np.ndarray | None = None      # (N,) uint8
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    def copy(self) -> "Scene":
        def c(a):
            return None if a is None else a.copy()
        return Scene(c(self.pos), c(self.vel), c(self.goal), c(self.radius),
                     c(self.max_speed), c(self.type),
                     dataclasses.replace(self.params), c(self.route),
                     c(self.waypoints), c(self.wp_idx), self.name)

    def subset(self, idx: np.ndarray) -> "Scene":
        """Scene made of the agents ``idx`` (routes keep their rows)."""
        s = self.copy()
        s.pos, s.vel, s.goal = s.pos[idx], s.vel[idx], s.goal[idx]
        s.radius, s.max_speed, s.type = s.radius[idx], s.max_speed[idx], s.type[idx]
        if s.route is not None:
            s.route, s.wp_idx = s.route[idx], s.wp_idx[idx]
        return s


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _agents(pos, goal, types, params, name, route=None, waypoints=None):
    n = pos.shape[0]
    types = np.asarray(types, dtype=np.uint8)
    radius = np.where(types == VEHICLE, 1.5, 0.5).astype(np.float32)
    vmax = np.where(types == VEHICLE, 5.0, 1.5).astype(np.float32)
    wp_idx = None
    if route is not None:
        route = np.ascontiguousarray(route, dtype=np.int32)
        wp_idx = np.zeros(n, dtype=np.uint8)
        waypoints = _f32(waypoints)
    return Scene(_f32(pos), np.zeros((n, 2), np.float32), _f32(goal), radius,
                 vmax, types, params, route, waypoints, wp_idx, name)


def open_square(n: int = 1000, side: float = 50.0, seed: int = 0) -> Scene:
    """Plain ORCA in an open square: 1,000 pedestrians in 50 x 50 m.

    Draw order: positions U([0,side]^2), then goals U([0,side]^2).  Radius
    0.5 m, max speed 1.5 m/s, initial velocity 0.  Uniform placement overlaps
    a few hundred pairs at t = 0, which exercises the overlap branch.
    """
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, side, size=(n, 2))
    goal = rng.uniform(0.0, side, size=(n, 2))
    p = OrcaParams(origin=(0.0, 0.0), extent=(side, side), cell_size=2.0)
    return _agents(pos, goal, np.zeros(n), p, f"open_square_{n}")


def shared_space(n_ped: int = 64000, n_veh: int = 1000, side: float = 500.0,
                 seed: int = 1) -> Scene:
    """Two counter-flowing pedestrian streams crossing vehicle lanes.

    Draw order: southbound stream (x, y, goal x, goal y), northbound stream
    (x, y, goal x, goal y), then vehicles (x jitter, y jitter, goal jitter).
    Streams occupy x in [0.4, 0.6] * side and start in opposite y-halves with
    goals on the far edge (the paper's two-way crossing, Sec. 4).  Vehicles
    drive in 10 east-west lanes, alternating direction, evenly spaced along
    the lane with uniform jitter; goal = the lane's far end with jitter.
    """
    rng = np.random.default_rng(seed)
    half = n_ped // 2
    rest = n_ped - half
    x0, x1 = 0.4 * side, 0.6 * side
    # southbound: start in the northern half, goal at the southern edge
    sx = rng.uniform(x0, x1, size=half)
    sy = rng.uniform(0.52 * side, side, size=half)
    sgx = rng.uniform(x0, x1, size=half)
    sgy = rng.uniform(0.0, 0.08 * side, size=half)
    # northbound: start in the southern half, goal at the northern edge
    nx_ = rng.uniform(x0, x1, size=rest)
    ny_ = rng.uniform(0.0, 0.48 * side, size=rest)
    ngx = rng.uniform(x0, x1, size=rest)
    ngy = rng.uniform(0.92 * side, side, size=rest)
    lanes = 10
    per_lane = n_veh // lanes if n_veh >= lanes else n_veh
    lane_id = np.arange(n_veh) % lanes
    slot = np.arange(n_veh) // lanes
    spacing = side / max(per_lane, 1)
    vjx = rng.uniform(-0.1 * spacing, 0.1 * spacing, size=n_veh)
    vjy = rng.uniform(-0.5, 0.5, size=n_veh)
    gj = rng.uniform(0.0, 0.02 * side, size=n_veh)
    lane_y = (lane_id + 0.5) * side / lanes
    vx = (slot + 0.5) * spacing + vjx
    vy = lane_y + vjy
    east = (lane_id % 2) == 0
    vgx = np.where(east, side - gj, gj)
    vgy = lane_y
    pos = np.concatenate([np.stack([sx, sy], 1), np.stack([nx_, ny_], 1),
                          np.stack([vx, vy], 1)])
    goal = np.concatenate([np.stack([sgx, sgy], 1), np.stack([ngx, ngy], 1),
                           np.stack([vgx, vgy], 1)])
    types = np.concatenate([np.zeros(n_ped), np.ones(n_veh)])
    p = OrcaParams(origin=(0.0, 0.0), extent=(side, side), cell_size=4.0)
    return _agents(pos, goal, types, p, f"shared_space_{n_ped}_{n_veh}")


def clusters(n: int = 1_000_000, side: float = 2000.0, n_clusters_axis: int = 8,
             sigma: float = 20.0, vehicle_every: int = 100, seed: int = 2) -> Scene:
    """Stress scene: agents in Gaussian clusters, goals at the opposite cluster.

    Draw order: lattice jitter of the cluster centres (x, y), then the
    agents' offsets N(0, sigma^2 I).  Agent i belongs to cluster i mod C; every
    ``vehicle_every``-th agent is a vehicle.  The goal is the centre of the
    point-reflected cluster (a, b) -> (A-1-a, A-1-b) plus the agent's own
    offset.  Peak density is high enough that many velocity LPs are empty and
    take the least-penetration fallback (Sec. 3).
    """
    rng = np.random.default_rng(seed)
    a_ = n_clusters_axis
    cell = side / a_
    jit = rng.uniform(-0.1 * cell, 0.1 * cell, size=(a_, a_, 2))
    ia, ib = np.meshgrid(np.arange(a_), np.arange(a_), indexing="ij")
    centres = np.stack([(ia + 0.5) * cell, (ib + 0.5) * cell], -1) + jit
    centres = centres.reshape(-1, 2)
    nc = a_ * a_
    cid = np.arange(n) % nc
    off = rng.normal(0.0, sigma, size=(n, 2))
    pos = centres[cid] + off
    ca, cb = cid // a_, cid % a_
    opp = (a_ - 1 - ca) * a_ + (a_ - 1 - cb)
    goal = centres[opp] + off
    types = (np.arange(n) % vehicle_every == 0).astype(np.uint8)
    p = OrcaParams(origin=(0.0, 0.0), extent=(side, side), cell_size=1.0)
    return _agents(pos, goal, types, p, f"clusters_{n}")


def batched_sizes(n_scenes: int = 512, lo: int = 100, hi: int = 20000,
                  seed: int = 3) -> np.ndarray:
    """Scene sizes log-uniform in [lo, hi] (first draws of the batched family)."""
    rng = np.random.default_rng(seed)
    return np.round(np.exp(rng.uniform(math.log(lo), math.log(hi),
                                       size=n_scenes))).astype(np.int64)


def batched(n_scenes: int = 512, lo: int = 100, hi: int = 20000,
            density: float = 0.5, vehicle_frac: float = 0.05,
            seed: int = 3) -> list[Scene]:
    """Independent scenes of uneven size for the batched path.

    Draw order: all sizes first (log-uniform), then for each scene in turn its
    positions and goals, both uniform in its square of side sqrt(n / density).
    The first round(vehicle_frac * n) agents of each scene are vehicles.
    """
    rng = np.random.default_rng(seed)
    sizes = np.round(np.exp(rng.uniform(math.log(lo), math.log(hi),
                                        size=n_scenes))).astype(np.int64)
    out = []
    for s, ns in enumerate(sizes):
        ns = int(ns)
        side = math.sqrt(ns / density)
        pos = rng.uniform(0.0, side, size=(ns, 2))
        goal = rng.uniform(0.0, side, size=(ns, 2))
        nv = int(round(vehicle_frac * ns))
        types = np.zeros(ns)
        types[:nv] = 1
        p = OrcaParams(origin=(0.0, 0.0), extent=(side, side), cell_size=4.0)
        out.append(_agents(pos, goal, types, p, f"batched_{s}_{ns}"))
    return out


def waypoint_square(n_ped: int = 4000, n_veh: int = 64, side: float = 100.0,
                    n_wp: int = 8, seed: int = 4) -> Scene:
    """Adjoint rollout scene: pedestrians and waypoint-following vehicles.

    Draw order: all positions U([0,side]^2), pedestrian goals U([0,side]^2),
    then the vehicles' waypoints U([0,side]^2), shape (n_veh, n_wp, 2).
    Vehicles are the last ``n_veh`` agents; vehicle v follows route v and
    its goal (used by the loss) is its last waypoint.
    """
    rng = np.random.default_rng(seed)
    n = n_ped + n_veh
    pos = rng.uniform(0.0, side, size=(n, 2))
    pgoal = rng.uniform(0.0, side, size=(n_ped, 2))
    wps = rng.uniform(0.0, side, size=(n_veh, n_wp, 2))
    goal = np.concatenate([pgoal, wps[:, -1, :]])
    types = np.concatenate([np.zeros(n_ped), np.ones(n_veh)])
    route = np.full(n, -1, dtype=np.int32)
    route[n_ped:] = np.arange(n_veh, dtype=np.int32)
    p = OrcaParams(origin=(0.0, 0.0), extent=(side, side), cell_size=2.0)
    return _agents(pos, goal, types, p, f"waypoint_square_{n}", route, wps)


# The five workloads at the sizes the paper-shaped benchmarks use.
WORKLOADS = {
    "open_square_1k": dict(fn="open_square", steps=100),
    "shared_space_65k": dict(fn="shared_space", steps=200),
    "clusters_1m": dict(fn="clusters", steps=50),
    "batched_512": dict(fn="batched", steps=50),
    "waypoint_square_4k": dict(fn="waypoint_square", steps=40),
}
