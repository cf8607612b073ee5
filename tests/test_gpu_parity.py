"""GPU path vs the CPU oracle, through the C ABI (needs a GB300).

Bar: bit-exact ROS tables (binary64 and the fixed-point increments), bit-exact
ignition steps, scars, work counts and burn-probability counts.  Cases span
several CTAs' worth of replicas, ragged grid widths (not multiples of the
32-cell plane words), borders and corners, non-fuel and harvested cells,
every fuel code, noise, thresholds, delta burn-out and clock lengths.
"""
import numpy as np
import pytest

import c2f_synth as S
import oracle
import paper_1905_09317_gb300 as c2f

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c2f.build()
    with c2f.Context(0) as c:
        yield c


def gpu_params(**kw):
    p = dict(kw)
    p.setdefault("outputs", c2f.OUT_SCARS | c2f.OUT_COUNTERS | c2f.OUT_IGN_STEPS)
    keys = {f[0] for f in c2f.SimParams._fields_}
    return c2f.default_params(**{k: v for k, v in p.items() if k in keys})


def load(ctx, w):
    L = w.landscape
    lid = ctx.load_landscape(L.fuel, L.slope, L.aspect, L.unburnable, L.cell_size)
    ctx.set_weather(lid, w.weather)
    return lid


def make_oracle(w, **over):
    L = w.landscape
    p = dict(w.params)
    p.update(over)
    return oracle.Oracle(L.fuel, L.slope, L.aspect, L.unburnable, cell_size=L.cell_size,
                         weather=w.weather, **p)


def run_gpu(ctx, w, **over):
    p = dict(w.params)
    p.update(over)
    lid = load(ctx, w)
    gp = gpu_params(**p)
    sid = ctx.simulate(lid, gp)
    n = w.landscape.fuel.size
    R = gp.n_replicas
    scars, ign = ctx.get_scars(sid, R, n, ign_steps=True)
    work, nign, cells = ctx.get_counters(sid, R)
    counts = ctx.burn_prob(sid, n)
    ctx.release(sid)
    ctx.release(lid)
    return dict(scars=scars, ign=ign, work=work, n_ignited=nign, ign_cell=cells, counts=counts)


def compare_replicas(w, g, replicas, **over):
    o = make_oracle(w, **over)
    for r in replicas:
        ref = o.run_replica(r)
        assert g["ign_cell"][r] == ref["ignition_cell"], r
        assert np.array_equal(g["ign"][r], ref["ign"].ravel()), f"ignition steps differ, replica {r}"
        assert np.array_equal(g["scars"][r], ref["scar"].ravel()), r
        assert g["work"][r] == ref["work"], (r, g["work"][r], ref["work"])
        assert g["n_ignited"][r] == ref["n_ignited"], r


# ------------------------------------------------------------------ K1
@pytest.mark.parametrize("ellipse_mode", [0, 1])
def test_ros_table_bit_exact(ctx, ellipse_mode):
    w = S.config2(side=67, n_replicas=1, hours=5)   # ragged width, all fuels, slopes
    w.landscape.fuel[3, 3] = 10                        # M2
    w.landscape.fuel[4, 4] = 12                        # O1b
    w.landscape.fuel[5, 5] = 5                         # C5
    w.landscape.fuel[6, 6] = 14                        # S2
    w.landscape.fuel[7, 7] = 15                        # S3
    w.landscape.unburnable = np.zeros_like(w.landscape.fuel)
    w.landscape.unburnable[10:12, 20:40] = 1
    w.weather[2, 0] = 55.0                             # high-wind branch
    lid = load(ctx, w)
    o = make_oracle(w, ellipse_mode=ellipse_mode, m1_pc=35.0, o1_curing_pct=45.0)
    gp = gpu_params(**dict(w.params, ellipse_mode=ellipse_mode, m1_pc=35.0, o1_curing_pct=45.0))
    n = w.landscape.fuel.size
    for h in range(5):
        ros8, hros, base = ctx.get_ros(lid, gp, h, n)
        for cell in range(n):
            row = o.cell_row(cell, h)
            b, hr = o.base_inc(cell, h)
            assert np.array_equal(ros8[cell], row["ros8"]), (h, cell, ros8[cell], row["ros8"])
            assert hros[cell] == row["hros"] and hr == row["hros"]
            assert np.array_equal(base[cell], b), (h, cell)
    ctx.release(lid)


def test_ros_table_const_rate(ctx):
    w = S.config1()
    lid = load(ctx, w)
    gp = gpu_params(**dict(w.params, const_ros=10.0, minutes_per_step=3))
    ros8, hros, base = ctx.get_ros(lid, gp, 0, 1600)
    assert np.all(ros8 == 10.0) and np.all(hros == 10.0)
    assert np.all(base == 30 * 2 ** 32)
    ctx.release(lid)


# ------------------------------------------------------------------ whole runs
def test_config1_full(ctx):
    w = S.config1()
    g = run_gpu(ctx, w)
    compare_replicas(w, g, [0])
    assert np.array_equal(g["counts"], g["scars"][0].astype(np.uint32))


@pytest.mark.parametrize("name", ["hand_3x3.txt", "hand_5x5.txt", "hand_wind_eq1_5x5.txt",
                                  "hand_wind_ray_5x5.txt", "hand_delta_5x5.txt",
                                  "hand_threshold_5x5.txt", "hand_burnhours_3x3.txt",
                                  "hand_clock5_3x3.txt", "hand_harvested_5x5.txt"])
def test_hand_enumeration(ctx, name):
    """Ignition steps and work count of hand-enumerated grids: constant rates
    on all axes, an ellipse (H, B, LB) under wind by Eq. (1) and by the ray of
    ellipse_mode 1, burn-out below delta, rejected messages under a receive
    threshold, a fire that burns one hour a day, a 5-minute clock and a
    harvested column (tests/golden/)."""
    from conftest import read_golden_grid
    meta, grid = read_golden_grid(name)
    gr = np.array(grid)
    rows, cols = gr.shape
    unb = None
    if "harvested_col" in meta:
        unb = np.zeros((rows, cols), np.uint8)
        unb[:, int(meta["harvested_col"])] = 1
    w = S.Workload(S.Landscape(np.ones((rows, cols), np.uint8), np.zeros((rows, cols), np.float32),
                               np.zeros((rows, cols), np.float32), unburnable=unb),
                   S.constant_weather(int(meta["hours"]), ws=0.0,
                                      wd_from=float(meta.get("wd_from", 270.0))),
                   dict(hours=int(meta["hours"]), ignition_cell=(rows // 2) * cols + cols // 2,
                        const_ros=float(meta["const_ros"]),
                        const_bros=float(meta.get("const_bros", 0.0)),
                        const_lb=float(meta.get("const_lb", 0.0)),
                        ellipse_mode=int(meta.get("ellipse_mode", 0)),
                        burnout_delta=float(meta.get("burnout_delta", 0.0)),
                        ros_threshold=float(meta.get("ros_threshold", 0.0)),
                        burn_hours_min=int(meta.get("burn_hours_min", 0)),
                        burn_hours_max=int(meta.get("burn_hours_max", 0)),
                        minutes_per_step=int(meta.get("minutes_per_step", 1))))
    g = run_gpu(ctx, w)
    assert np.array_equal(g["ign"][0].reshape(rows, cols), gr)
    assert g["work"][0] == int(meta["work"])
    assert g["n_ignited"][0] == int((gr >= 0).sum())


@pytest.mark.parametrize("seed", range(16))
def test_random_small_cases(ctx, seed):
    w = S.random_small_case(seed)
    if not (w.landscape.fuel != 0).any():
        pytest.skip("no fuel")
    unb = w.landscape.unburnable
    burnable = (w.landscape.fuel != 0) & (unb == 0 if unb is not None else True)
    if not burnable.any():
        pytest.skip("no burnable cell")
    R = 37
    g = run_gpu(ctx, w, n_replicas=R)
    compare_replicas(w, g, range(R))
    assert np.array_equal(g["counts"], g["scars"].sum(0).astype(np.uint32))


def test_edges_corners_and_strips(ctx):
    cases = []
    for rows, cols, cell in [(1, 1, 0), (1, 45, 0), (45, 1, 44), (7, 33, 0), (7, 33, 7 * 33 - 1),
                             (9, 64, 63), (3, 97, 96)]:
        fuel = np.full((rows, cols), 2, np.uint8)
        w = S.Workload(S.Landscape(fuel, np.zeros_like(fuel, np.float32),
                                   np.zeros_like(fuel, np.float32)),
                       S.weather_stream(3, seed=rows * cols),
                       dict(hours=3, ignition_cell=cell, ros_sigma=0.1, seed=11))
        cases.append(w)
    for w in cases:
        g = run_gpu(ctx, w, n_replicas=3)
        compare_replicas(w, g, range(3))


def test_maximum_side_strips(ctx):
    """Strips at the largest side the boundary accepts (65,535 cells): cell ids,
    packed (row, col) coordinates and plane words at their limits, with most of
    the grid outside the shared-memory window of the bit planes, which the fire
    leaves; ignition in the last row or column.  A side of 65,536 is rejected."""
    # wind from the far end of each strip (east of the row strip, south of the
    # column strip): the head fire runs back along it from its last cells
    for rows, cols, cell, wd_from in [(3, 65535, 2 * 65535 - 1, 90.0), (65535, 3, 3 * 65535 - 2, 180.0)]:
        fuel = np.full((rows, cols), 2, np.uint8)           # C2
        zeros = np.zeros_like(fuel, np.float32)
        w = S.Workload(S.Landscape(fuel, zeros, zeros),
                       S.constant_weather(12, ws=30.0, wd_from=wd_from, ffmc=93.0, bui=100.0),
                       dict(hours=12, ignition_cell=cell, ros_sigma=0.1, seed=13))
        g = run_gpu(ctx, w, n_replicas=2)
        # the fire runs about 300 cells along the strip: past the 256-cell window
        assert g["n_ignited"].min() > 800
        compare_replicas(w, g, range(2))
    for shape in [(1, 65536), (65536, 1)]:
        with pytest.raises(c2f.C2FError) as e:
            ctx.load_landscape(np.full(shape, 2, np.uint8))
        assert e.value.code == c2f.C2F_EINVAL


def test_clock_lengths_and_options(ctx):
    w = S.config2(side=48, n_replicas=24, hours=4)
    for over in (dict(minutes_per_step=60), dict(minutes_per_step=5), dict(ros_threshold=3.0),
                 dict(burnout_delta=2.0), dict(ellipse_mode=1), dict(ros_sigma=1.0),
                 dict(ignition_mode=0, ignition_cell=int(np.flatnonzero(w.landscape.fuel.ravel())[7]))):
        g = run_gpu(ctx, w, **over)
        compare_replicas(w, g, range(24), **over)


def test_capacity_overflow_rerun_gives_same_result(ctx):
    w = S.config2(side=96, n_replicas=40, hours=6)
    ref = run_gpu(ctx, w)
    ctx.set_list_capacity(8)
    try:
        small = run_gpu(ctx, w)
    finally:
        ctx.set_list_capacity(0)
    for k in ("ign", "scars", "work", "n_ignited", "counts"):
        assert np.array_equal(ref[k], small[k]), k
    compare_replicas(w, small, range(0, 40, 5))


def test_burn_prob_matches_oracle_sum(ctx):
    w = S.config2(side=128, n_replicas=64, hours=6)
    g = run_gpu(ctx, w)
    o = make_oracle(w)
    scars = np.stack([o.run_replica(r)["scar"].ravel() for r in range(64)])
    assert np.array_equal(g["counts"], oracle.burn_prob(scars))


def test_batch_equals_separate_runs(ctx):
    ws = [S.config2(side=s, n_replicas=r, hours=h) for s, r, h in ((40, 5, 3), (70, 33, 4), (33, 2, 2))]
    ws[1].params["seed"] = 77
    lids = [load(ctx, w) for w in ws]
    ps = [gpu_params(**w.params) for w in ws]
    sids = ctx.simulate_batch(lids, ps)
    for w, lid, sid, p in zip(ws, lids, sids, ps):
        n = w.landscape.fuel.size
        scars, ign = ctx.get_scars(sid, p.n_replicas, n, ign_steps=True)
        work, _, _ = ctx.get_counters(sid, p.n_replicas)
        alone = run_gpu(ctx, w)
        assert np.array_equal(ign, alone["ign"]) and np.array_equal(work, alone["work"])
        ctx.release(sid)
    for lid in lids:
        ctx.release(lid)


def test_config2_full_size_sampled_replicas(ctx):
    """512x512, 1000 replicas, 24 h, one c2f_simulate (the library's default
    launch sizing, the benchmark's plain steps); every 125th replica is
    replayed by the oracle, ignition steps included."""
    w = S.config2()
    g = run_gpu(ctx, w)
    compare_replicas(w, g, range(0, 1000, 125))
    assert np.array_equal(g["counts"], g["scars"].sum(0, dtype=np.uint32))
    assert g["counts"].max() <= 1000


def test_errors(ctx):
    w = S.config1()
    lid = load(ctx, w)
    with pytest.raises(c2f.C2FError) as e:
        ctx.simulate(lid, gpu_params(hours=11))          # weather is 10 h long
    assert e.value.code == c2f.C2F_EINVAL
    with pytest.raises(c2f.C2FError) as e:
        ctx.simulate(lid, gpu_params(minutes_per_step=7))
    assert e.value.code == c2f.C2F_EINVAL
    with pytest.raises(c2f.C2FError) as e:
        ctx.simulate(lid, gpu_params(ros_sigma=2.0))
    assert e.value.code == c2f.C2F_EINVAL
    with pytest.raises(c2f.C2FError) as e:
        ctx.simulate(12345, gpu_params())
    assert e.value.code == c2f.C2F_ENOTFOUND
    bad = np.full((4, 4), 16, np.uint8)
    with pytest.raises(c2f.C2FError) as e:
        ctx.load_landscape(bad)
    assert e.value.code == c2f.C2F_EINVAL
    fuel = np.zeros((4, 4), np.uint8); fuel[0, 0] = 1
    l2 = ctx.load_landscape(fuel)
    ctx.set_weather(l2, S.constant_weather(1))
    with pytest.raises(c2f.C2FError) as e:
        ctx.simulate(l2, gpu_params(ignition_cell=5))    # non-fuel ignition
    assert e.value.code == c2f.C2F_EINVAL
    ctx.release(l2)
    ctx.release(lid)


def test_autotune_keeps_results(ctx):
    """Every knob the autotuner turns (warps per CTA, shared / global lists,
    shared-memory sizing, compaction trigger, list capacity) changes speed
    only: the ignition steps are the same under each setting it tries and
    under the one it keeps."""
    ws = [S.config2(side=s, n_replicas=r, hours=3) for s, r in ((60, 30), (90, 12))]
    lids = [load(ctx, w) for w in ws]
    ps = [gpu_params(**w.params) for w in ws]

    def steps():
        return [ctx.get_scars(sid, p.n_replicas, w.landscape.fuel.size, ign_steps=True)[1]
                for sid, p, w in zip(ctx.simulate_batch(lids, ps), ps, ws)]

    before = steps()
    t = ctx.autotune_full(lids, ps, sample_replicas=16)
    assert t["threads"] in (32, 64, 128) and t["smem_lists"] in (0, 1) and t["frontier_ms"] > 0
    assert t["compact_eighths"] in (4, 6, 7) and t["warps_per_sm"] in (0, 4, 6, 8, 11)
    assert t["list_capacity"] >= 0 and t["candidates"] >= 7
    for a, b in zip(before, steps()):
        assert np.array_equal(a, b)
    # each knob on its own, including settings that force list overflows and re-runs
    settings = [dict(threads=64, smem=1), dict(threads=32, smem=0), dict(threads=128, smem=11),
                dict(threads=32, smem=4, eighths=2), dict(threads=32, smem=1, eighths=7),
                dict(threads=32, smem=0, cap=64), dict(threads=128, smem=0, cap=16, eighths=4)]
    for st in settings:
        ctx.set_frontier_config(st["threads"], st["smem"])
        ctx.set_compaction(st.get("eighths", 6))
        ctx.set_list_capacity(st.get("cap", 0))
        for a, b in zip(before, steps()):
            assert np.array_equal(a, b), st
    threads, smem, ms = ctx.autotune(lids, ps, sample_replicas=16)
    assert threads in (32, 64, 128) and smem in (0, 1, 4, 6, 8, 11) and ms > 0
    ctx.set_frontier_config(32, 1)
    ctx.set_compaction(6)
    ctx.set_list_capacity(0)
