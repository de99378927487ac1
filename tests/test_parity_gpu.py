"""CUDA path against the FP64 oracle, element by element (needs a GPU).

Every case runs one synchronous step (or a per-step rollout) on the GPU
through the C ABI and the same step in the oracle from the identical FP32
state, then checks cells, neighbour lists and waypoint indices bit for bit
and velocities/positions within the stated tolerances (parity_util).
"""
import numpy as np
import pytest

import oracle
from paper_2008_11578_gb300 import api, scenes
from tests.parity_util import cells_oracle as _cells_oracle
from tests.parity_util import compare, gpu_step

pytestmark = pytest.mark.gpu


def test_open_square_one_step():
    s = scenes.open_square()
    g = gpu_step(s)
    assert g["status"] == 0
    assert np.array_equal(g["cell"], _cells_oracle(s))
    st = compare(s, g)
    assert st["infeasible_oracle"] > 100   # uniform spawn overlaps: fallback exercised


def test_open_square_per_step_rollout():
    """Per-step parity from identical states along a 40-step GPU rollout."""
    s = scenes.open_square()
    for t in range(40):
        g = gpu_step(s)
        compare(s, g)
        s.pos, s.vel = g["pos"], g["vel"]


def test_shared_space_small():
    s = scenes.shared_space(n_ped=6400, n_veh=100, side=160.0)
    for t in range(3):
        g = gpu_step(s)
        assert np.array_equal(g["cell"], _cells_oracle(s))
        compare(s, g)
        s.pos, s.vel = g["pos"], g["vel"]


def test_clusters_dense_sampled():
    """Density of the 1M-agent cluster workload (15,625 agents per cluster),
    four clusters; oracle on a sample that includes every fallback agent."""
    s = scenes.clusters(n=62500, side=500.0, n_clusters_axis=2)
    g = gpu_step(s)
    rng = np.random.default_rng(0)
    inf = np.nonzero(g["flags"] & 1)[0]
    sel = np.unique(np.concatenate([rng.choice(s.n, 6000, replace=False),
                                    rng.choice(inf, min(4000, len(inf)), replace=False)]))
    assert np.array_equal(g["cell"], _cells_oracle(s))
    st = compare(s, g, sel=sel)
    assert st["infeasible_oracle"] > 1000


def test_clusters_full_size_sampled():
    """The 1M-agent workload at full size in the library's default launch
    shape (the benchmark's shape is in test_full_size_gpu.py); the oracle
    computes 3,000 sampled agents one by one."""
    s = scenes.clusters()
    g = gpu_step(s)
    rng = np.random.default_rng(1)
    sel = np.sort(rng.choice(s.n, 3000, replace=False))
    assert np.array_equal(g["cell"], _cells_oracle(s))
    compare(s, g, sel=sel)


def test_waypoints_rollout():
    s = scenes.waypoint_square()
    for t in range(6):
        g = gpu_step(s)
        compare(s, g)
        s.pos, s.vel, s.wp_idx = g["pos"], g["vel"], g["wp_idx"]


def test_vpref_delta():
    s = scenes.open_square(400, 30.0, seed=3)
    d = np.random.default_rng(2).normal(0, 0.3, (1, s.n, 2)).astype(np.float32)
    g = gpu_step(s, vpref_delta=d)
    compare(s, g, vpref_delta=d[0])


def test_results_independent_of_cell_and_block_size():
    """The neighbour search is exact, so the grid (square or rectangular
    cells) and launch shape change nothing: outputs are bitwise identical."""
    s = scenes.open_square(1500, 60.0, seed=4)
    ref = gpu_step(s, n_steps=3)
    for c, h, b in [(0.7, None, 0), (5.0, None, 64), (13.0, None, 32), (61.0, None, 96),
                    (2.0, None, 128), (4.0, 0.5, 64), (0.5, 4.0, 128), (30.0, 0.25, 64),
                    (1.0, 61.0, 32)]:
        g = gpu_step(s, n_steps=3, cell_size=c, cell_height=h, block_size=b)
        assert np.array_equal(g["pos"], ref["pos"]) and np.array_equal(g["vel"], ref["vel"])
        assert np.array_equal(g["nbr"], ref["nbr"])
        g1 = gpu_step(s, cell_size=c, cell_height=h, block_size=b)   # cells of step 1
        assert np.array_equal(g1["cell"], _cells_oracle(s, c, h))


@pytest.mark.parametrize("w,h", [(4.0, 0.5), (2.0, 0.375), (0.5, 0.5), (8.0, 1.0)])
def test_rectangular_cells_at_cluster_density(w, h):
    """Thin, wide cells (the search's preferred shape) at the density of the
    1M-agent workload: cells and neighbour lists bit-exact, velocities and
    positions within tolerance, on a sample with every fallback agent."""
    s = scenes.clusters(n=62500, side=500.0, n_clusters_axis=2)
    g = gpu_step(s, cell_size=w, cell_height=h, block_size=64)
    assert g["status"] == 0
    assert np.array_equal(g["cell"], _cells_oracle(s, w, h))
    rng = np.random.default_rng(5)
    inf = np.nonzero(g["flags"] & 1)[0]
    sel = np.unique(np.concatenate([rng.choice(s.n, 3000, replace=False),
                                    rng.choice(inf, min(2000, len(inf)), replace=False)]))
    compare(s, g, sel=sel)


def test_multi_step_call_equals_single_steps_and_is_deterministic():
    s = scenes.open_square(800, 40.0, seed=8)
    a = gpu_step(s, n_steps=5)
    b = gpu_step(s, n_steps=5)
    assert np.array_equal(a["pos"], b["pos"]) and np.array_equal(a["vel"], b["vel"])
    c = s.copy()
    for _ in range(5):
        g = gpu_step(c)
        c.pos, c.vel = g["pos"], g["vel"]
    assert np.array_equal(a["pos"], c.pos) and np.array_equal(a["vel"], c.vel)


def test_repeated_calls_bin_in_the_recorded_order_and_change_nothing():
    # the last step of a call records its sorted order; the next call bins in
    # that order, which must not change any result
    import torch
    s = scenes.open_square(3000, 80.0, seed=21)
    a = gpu_step(s, n_steps=4, debug=False)
    ds = api.DeviceScene(s, "cuda")
    for _ in range(4):
        ds.step(1)
    torch.cuda.synchronize()
    assert ds.sync_status() == 0
    assert np.array_equal(ds.pos.cpu().numpy(), a["pos"])
    assert np.array_equal(ds.vel.cpu().numpy(), a["vel"])
    # the caller reorders its agents between calls: the recorded order is
    # then an arbitrary permutation, still a valid one
    perm = np.random.default_rng(3).permutation(s.n)
    pt = torch.as_tensor(perm, device="cuda")
    for t in (ds.pos, ds.vel, ds.goal, ds.radius, ds.max_speed, ds.type):
        t.copy_(t[pt].clone())
    c = s.copy()
    c.pos, c.vel = a["pos"], a["vel"]
    c = c.subset(perm)
    ds.step(1)
    torch.cuda.synchronize()
    b = gpu_step(c, debug=False)
    assert ds.sync_status() == 0
    assert np.array_equal(ds.pos.cpu().numpy(), b["pos"])
    assert np.array_equal(ds.vel.cpu().numpy(), b["vel"])
    ds.close()


# ------------------------------------------------------------ edge cases ----

def test_empty_scene():
    s = scenes.open_square(0, 10.0)
    g = gpu_step(s)
    assert g["status"] == 0 and g["pos"].shape == (0, 2)


def test_single_agent_moves_to_goal():
    s = scenes.open_square(1, 10.0, seed=9)
    g = gpu_step(s)
    compare(s, g)


def test_k_zero_and_k_32():
    # 16 and 17 straddle the LP's constraint order (all lines sorted by
    # penetration up to 16 lines, only the two most violated first above)
    for k in (0, 1, 16, 17, 32):
        s = scenes.open_square(700, 30.0, seed=10)
        s.params.max_neighbors = k
        g = gpu_step(s)
        compare(s, g)


def test_k_16_with_vehicle_kinematic_lines():
    """k = 16: pedestrians' 16 half-planes take the sorted constraint order,
    a vehicle's 16 + 3 kinematic half-planes take the two-most-violated
    order."""
    s = scenes.shared_space(n_ped=3000, n_veh=200, side=90.0, seed=15)
    s.params.max_neighbors = 16
    s.params.vehicle_turn_rate, s.params.vehicle_accel = 0.8, 2.0
    g = gpu_step(s)
    assert g["status"] == 0
    compare(s, g, sel=np.arange(0, s.n, 2))


def test_grid_at_the_cell_limit():
    """8192 x 8192 = 2^26 cells (ORCA_MAX_CELLS): the binning kernel's scan
    then runs over 67M counters in the largest per-block ranges; 20,000
    agents spread over the grid and a dense patch, sampled against the
    oracle, all cells bit-exact."""
    s = scenes.open_square(20000, 2048.0, seed=13)
    rng = np.random.default_rng(13)
    s.pos[:5000] = (1000.0 + 30.0 * rng.random((5000, 2))).astype(np.float32)   # dense patch
    cell = 0.25
    assert s.params.grid_dims(cell) == (8192, 8192)
    g = gpu_step(s, cell_size=cell)
    assert g["status"] == 0
    assert np.array_equal(g["cell"], _cells_oracle(s, cell))
    sel = np.unique(np.concatenate([np.arange(0, s.n, 13), np.arange(0, 5000, 5)]))
    compare(s, g, sel=sel)


def test_k_32_with_vehicle_kinematic_lines():
    """The largest shared-memory footprint: k = 32 neighbours plus the three
    kinematic half-planes of a vehicle (35 slots per thread, opt-in shared
    memory), blocks of 64 and 128."""
    s = scenes.shared_space(n_ped=6400, n_veh=300, side=120.0, seed=14)
    s.params.max_neighbors = 32
    s.params.vehicle_turn_rate, s.params.vehicle_accel = 0.8, 2.0
    for block in (64, 128):
        g = gpu_step(s, block_size=block)
        assert g["status"] == 0
        compare(s, g, sel=np.arange(0, s.n, 3))


def test_all_agents_in_one_cell_and_outside_box():
    s = scenes.open_square(600, 30.0, seed=11)
    g = gpu_step(s, cell_size=1000.0)
    compare(s, g)
    t = s.copy()
    t.pos = (t.pos * np.float32(2.0) - np.float32(20.0)).astype(np.float32)   # spills out of the box
    g = gpu_step(t)
    assert np.array_equal(g["cell"], _cells_oracle(t))
    compare(t, g)


def test_coincident_and_exact_ties():
    """Agents on an exact lattice (many equal keys, broken by index) and two
    agents at the same point."""
    xs = np.arange(12, dtype=np.float32)
    P = np.stack(np.meshgrid(xs, xs), -1).reshape(-1, 2).astype(np.float32)
    P = np.concatenate([P, P[:1]])          # one duplicate position
    n = len(P)
    s = scenes.Scene(P, np.zeros_like(P), P[::-1].copy(), np.full(n, 0.3, np.float32),
                     np.full(n, 1.5, np.float32), (np.arange(n) % 7 == 0).astype(np.uint8),
                     scenes.OrcaParams(extent=(12.0, 12.0), cell_size=1.0))
    g = gpu_step(s)
    compare(s, g)


def test_nonfinite_input_reports_status():
    s = scenes.open_square(50, 10.0, seed=12)
    s.pos[7, 0] = np.nan
    g = gpu_step(s)
    assert g["status"] == 4


def test_counting_variant_computes_the_same_step_and_consistent_tallies():
    """The counting variant (FLOP accounting and search tallies) is a
    separate instantiation of the solve kernel: it must compute the plain
    step bit for bit, and its tallies must fit together (every final list
    entry was admitted, a shift moves at most k - 1 entries per admission,
    every agent scans at least its own row, a loop iteration tests at most
    one candidate per cursor, and the phase clocks add up within the
    thread's total)."""
    import torch
    s = scenes.clusters(n=60000, side=500.0, n_clusters_axis=4, sigma=8.0, seed=31)
    plain = api.DeviceScene(s, "cuda")
    counted = api.DeviceScene(s, "cuda")
    c = torch.zeros(13, dtype=torch.int64, device="cuda")
    api.orca_scene_set_counters(counted.handle, c)
    plain.step(1)
    counted.step(1)
    torch.cuda.synchronize()
    assert torch.equal(plain.pos, counted.pos) and torch.equal(plain.vel, counted.vel)
    api.orca_scene_set_counters(counted.handle, None)
    dbg = api.DeviceScene(s, "cuda", debug=True)
    dbg.step(1)
    torch.cuda.synchronize()
    lists = int(dbg.dbg["cnt"].sum())
    k = int(s.params.max_neighbors)
    t = [int(x) for x in c.cpu().numpy()]
    n = s.n
    assert t[4] == n                         # agent updates
    assert t[1] == lists                     # half-planes built = list entries
    assert t[9] >= lists                     # admissions
    assert t[10] <= t[9] * (k - 1)           # shifts
    assert t[11] >= n                        # rows scanned
    assert 2 * t[12] >= t[0] and t[12] <= t[0] + 2 * t[11]   # two-cursor iterations
    assert 0 < t[5] and 0 < t[6] and 0 < t[7] and t[5] + t[6] + t[7] <= t[8]
    for ds in (plain, counted, dbg):
        ds.close()


def test_launch_count():
    s = scenes.open_square(100, 10.0)
    ds = api.DeviceScene(s)
    assert ds.launch_count(3) == 2 * 3   # binning + solve per step
    assert ds.launch_count(0) == 0
    ds.close()


def _full_speed_vehicle_apexes(count=24, seed=60):
    """Small groups, each a vehicle moving at exactly its maximum speed among
    pedestrians, kept only where the oracle's answer is the vehicle's own
    velocity: the apex of its f = 0 half-planes (car|person), which all pass
    through that velocity and here lie on the speed circle.  Groups sit 100 m
    apart, so they do not interact."""
    rng = np.random.default_rng(seed)
    groups = []
    while len(groups) < count:
        th = rng.uniform(0, 2 * np.pi)
        v0 = np.array([5.0 * np.cos(th), 5.0 * np.sin(th)], np.float32)
        if float(v0[0]) ** 2 + float(v0[1]) ** 2 <= 25.0:
            continue        # keep headings whose FP32 velocity is a hair outside the circle,
                            # as an earlier step's clip to max speed leaves it
        m = int(rng.integers(3, 7))
        P = np.concatenate([[[0.0, 0.0]], rng.uniform(-4, 4, (m, 2))]).astype(np.float32)
        V = np.concatenate([[v0], rng.normal(0, 1.0, (m, 2))]).astype(np.float32)
        G = np.concatenate([[[30 * np.cos(th + rng.normal(0, 0.5)), 30 * np.sin(th + rng.normal(0, 0.5))]],
                            rng.uniform(-10, 10, (m, 2))]).astype(np.float32)
        T = np.r_[1, np.zeros(m)].astype(np.uint8)
        s = scenes.Scene(P, V, G, np.where(T == 1, 1.5, 0.5).astype(np.float32),
                         np.where(T == 1, 5.0, 1.5).astype(np.float32), T,
                         scenes.OrcaParams(origin=(-50.0, -50.0), extent=(100.0, 100.0)))
        r = oracle.step(s, sel=np.array([0]))
        if (r.flags[0] & 1) == 0 and r.cnt[0] >= 2 and r.tstar[0] < -0.01 and \
                np.abs(r.vel[0] - V[0]).max() < 1e-5:
            groups.append(s)
    shift = [np.array([100.0 * q, 0.0], np.float32) for q in range(count)]
    cat = lambda f: np.concatenate([f(q, g) for q, g in enumerate(groups)])
    return scenes.Scene(cat(lambda q, g: g.pos + shift[q]), cat(lambda q, g: g.vel),
                        cat(lambda q, g: g.goal + shift[q]), cat(lambda q, g: g.radius),
                        cat(lambda q, g: g.max_speed), cat(lambda q, g: g.type),
                        scenes.OrcaParams(origin=(-50.0, -50.0),
                                          extent=(100.0 * count + 100.0, 100.0), cell_size=4.0))


def test_vehicle_at_full_speed_on_its_own_half_plane_apex():
    """The LP optimum at the apex of f = 0 half-planes on the speed circle is
    feasible (a rounding allowance keeps the 1D intervals from reading empty)."""
    s = _full_speed_vehicle_apexes()
    g = gpu_step(s)
    st = compare(s, g)
    veh = s.type == 1
    assert (g["flags"][veh] & 1).sum() == 0


@pytest.mark.parametrize("scheme", ["work_units", "warp"])
@pytest.mark.parametrize("name", ["open_square", "clusters", "shared_space"])
def test_cooperative_lp_matches_per_thread_lp(name, scheme):
    """The paper's block-cooperative work-unit LP and the warp-cooperative LP
    (the comparison variants) compute the same intervals as the per-thread LP
    (min and max are exact; only differently contracted multiply-adds round
    differently), so one step agrees to 1e-5; and they agree with the oracle
    like the per-thread LP does."""
    import torch
    s = {"open_square": lambda: scenes.open_square(3000, 80.0, seed=61),
         "clusters": lambda: scenes.clusters(n=62500, side=500.0, n_clusters_axis=2),
         "shared_space": lambda: scenes.shared_space(n_ped=6400, n_veh=100, side=160.0)}[name]()
    flag = {"work_units": api.LP_WORK_UNITS, "warp": api.LP_WARP}[scheme]
    out = {}
    for flags in (0, flag):
        ds = api.DeviceScene(s, "cuda", debug=True, flags=flags)
        ds.step(1)
        torch.cuda.synchronize()
        assert ds.sync_status() == 0
        out[flags] = (ds.pos.cpu().numpy(), ds.vel.cpu().numpy())
        ds.close()
    a, b = out[0], out[flag]
    assert np.abs(a[1].astype(np.float64) - b[1]).max() <= 1e-5
    assert np.abs(a[0].astype(np.float64) - b[0]).max() <= 1e-5
    g = gpu_step(s, flags=flag)
    compare(s, g, sel=np.arange(0, s.n, max(1, s.n // 3000)))


@pytest.mark.parametrize("name", ["open_square", "clusters", "shared_space", "kinematic"])
def test_enumeration_lp_matches_oracle(name):
    """Active-set enumeration (the second comparison scheme) builds every
    candidate optimum and keeps the best; it meets the oracle like the
    incremental LP does, on the feasible and the least-penetration path.
    Where the oracle finds the least-penetration minimiser ill-conditioned
    (condition number above 1e6: a bisector of two half-planes nearly
    tangent to the speed circle, or more than three planes through one
    point), the FP32 rim point is fixed only to about the square root of
    the rounding, so those agents are held to 1e-3 m/s instead; their
    neighbour lists stay exact."""
    s = {"open_square": lambda: scenes.open_square(3000, 80.0, seed=62),
         "clusters": lambda: scenes.clusters(n=62500, side=500.0, n_clusters_axis=2),
         "shared_space": lambda: scenes.shared_space(n_ped=6400, n_veh=100, side=160.0),
         "kinematic": lambda: scenes.shared_space(n_ped=6400, n_veh=300, side=160.0, seed=8)}[name]()
    if name == "kinematic":
        s.params.vehicle_turn_rate, s.params.vehicle_accel = 0.8, 2.0
    for t in range(2):
        g = gpu_step(s, flags=api.LP_ENUMERATION)
        assert g["status"] == 0
        sel = np.unique(np.concatenate([np.arange(0, s.n, max(1, s.n // 3000)),
                                        np.nonzero(g["flags"] & 1)[0][:2000]]))
        r = oracle.step(s, sel=sel)
        ill = r.cond > 1e6
        assert ill.mean() < 0.3   # the sample is weighted toward fallback agents
        st = compare(s, g, sel=sel[~ill])
        if name in ("open_square", "clusters"):
            assert st["infeasible_oracle"] > 100
        if ill.any():
            rb = oracle.step(s, sel=sel[ill])
            assert np.array_equal(g["nbr"][sel[ill]][:, :s.params.max_neighbors], rb.nbr)
            assert np.abs(g["vel"][sel[ill]].astype(np.float64) - rb.vel).max() <= 1e-3
        s.pos, s.vel = g["pos"], g["vel"]


@pytest.mark.parametrize("name", ["open_square", "clusters", "shared_space", "waypoints",
                                  "kinematic"])
def test_checked_mode_certifies_and_changes_nothing(name):
    """ORCA_DEBUG_CHECKED: every step certifies its k-lists, cell ranges and
    LP results on the device; on correct steps nothing is flagged (over four
    steps), and one step agrees with the plain step to FP32 rounding (the
    checked kernel is compiled separately, so multiply-adds may contract
    differently)."""
    import torch
    s = {"open_square": lambda: scenes.open_square(3000, 80.0, seed=63),
         "clusters": lambda: scenes.clusters(n=62500, side=500.0, n_clusters_axis=2),
         "shared_space": lambda: scenes.shared_space(n_ped=6400, n_veh=100, side=160.0),
         "waypoints": lambda: scenes.waypoint_square(n_ped=1500, n_veh=60, side=70.0, seed=9),
         "kinematic": lambda: scenes.shared_space(n_ped=6400, n_veh=300, side=160.0, seed=8)}[name]()
    if name == "kinematic":
        s.params.vehicle_turn_rate, s.params.vehicle_accel = 0.8, 2.0
    out = {}
    for flags in (0, api.CHECKED):
        ds = api.DeviceScene(s, "cuda", flags=flags)
        ds.step(1)
        torch.cuda.synchronize()
        assert ds.sync_status() == 0, flags
        out[flags] = (ds.pos.cpu().numpy(), ds.vel.cpu().numpy())
        ds.step(3)
        torch.cuda.synchronize()
        assert ds.sync_status() == 0, flags
        ds.close()
    assert np.abs(out[0][0].astype(np.float64) - out[api.CHECKED][0]).max() <= 1e-5
    assert np.abs(out[0][1].astype(np.float64) - out[api.CHECKED][1]).max() <= 1e-5


def test_save_and_resume_the_state():
    """The scene state lives in the caller's tensors: saving them
    (torch.save) and stepping a new scene from the saved copy reproduces the
    run bit for bit."""
    import io
    import torch
    s = scenes.waypoint_square(n_ped=1500, n_veh=60, side=70.0, seed=9)
    ds = api.DeviceScene(s, "cuda")
    ds.step(3)
    buf = io.BytesIO()
    torch.save({"pos": ds.pos, "vel": ds.vel, "wp_idx": ds.wp_idx}, buf)
    ds.step(4)
    torch.cuda.synchronize()
    a = [t.cpu().numpy() for t in (ds.pos, ds.vel, ds.wp_idx)]
    ds.close()
    buf.seek(0)
    saved = torch.load(buf)
    ds2 = api.DeviceScene(s, "cuda")
    ds2.set_state(pos=saved["pos"], vel=saved["vel"], wp_idx=saved["wp_idx"])
    ds2.step(4)
    torch.cuda.synchronize()
    assert ds2.sync_status() == 0
    for x, y in zip(a, (ds2.pos, ds2.vel, ds2.wp_idx)):
        assert np.array_equal(x, y.cpu().numpy())
    ds2.close()


@pytest.mark.parametrize("which", ["shared_space", "waypoints", "clusters"])
def test_vehicle_kinematic_limits(which):
    """Vehicles with turn-rate and acceleration limits (extra half-planes)
    against the oracle, per step along a short GPU rollout."""
    s = {"shared_space": lambda: scenes.shared_space(n_ped=6400, n_veh=300, side=160.0, seed=8),
         "waypoints": lambda: scenes.waypoint_square(n_ped=1500, n_veh=60, side=70.0, seed=9),
         "clusters": lambda: scenes.clusters(n=62500, side=500.0, n_clusters_axis=2,
                                             vehicle_every=20)}[which]()
    s.params.vehicle_turn_rate, s.params.vehicle_accel = 0.8, 2.0
    sel = None if s.n < 20000 else np.arange(0, s.n, 7)
    veh = s.type == 1
    for t in range(4):
        g = gpu_step(s)
        compare(s, g, sel=sel)
        if t == 0 and s.route is None:
            # from rest the speed along the preferred direction grows by at most
            # accel * dt = 0.5 m/s for vehicles whose LP is feasible (an empty LP
            # trades the limit against the ORCA half-planes); it binds somewhere
            ok = veh & ((g["flags"] & 1) == 0)
            h = (s.goal - s.pos)[ok].astype(np.float64)
            h /= np.linalg.norm(h, axis=1, keepdims=True)
            along = (g["vel"][ok].astype(np.float64) * h).sum(1)
            assert ok.sum() >= 1 and along.max() <= 0.5 + 1e-5
            assert (along > 0.5 - 1e-5).sum() >= 1
        s.pos, s.vel = g["pos"], g["vel"]
        if "wp_idx" in g:
            s.wp_idx = g["wp_idx"]
