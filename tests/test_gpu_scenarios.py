"""Weather scenarios on the GPU vs the oracle (needs a GB300).

Sec. 3.1, uncertainty source (3): a landscape carries several weather
streams with probabilities; each replica draws one (Philox counter
(replica, 0, 0, 2), thresholds T_s) and runs under it.  Checked bit for bit
against the oracle: every replica's drawn scenario, its ignition steps, work
and ignited counts, the stacked table rows of every scenario, and the burn
counts; a one-hot probability vector must reproduce the single-stream run of
that stream; batched and served runs must equal the plain ones.
"""
import numpy as np
import pytest

import c2f_synth as S
import oracle
import paper_1905_09317_gb300 as c2f

pytestmark = pytest.mark.gpu

_KEYS = {f[0] for f in c2f.SimParams._fields_}
_OUT = c2f.OUT_SCARS | c2f.OUT_COUNTERS | c2f.OUT_IGN_STEPS


def _params(**kw):
    kw.setdefault("outputs", _OUT)
    return c2f.default_params(**{k: v for k, v in kw.items() if k in _KEYS})


def _world(side=75, n_replicas=48, hours=4, n_scen=3, seed=31):
    w = S.config2(side=side, n_replicas=n_replicas, hours=hours)
    w.params["seed"] = seed
    w.params["ros_sigma"] = 0.1
    # streams of different wind strength and direction; scenario 0 is the base stream
    weathers = [w.weather] + [S.weather_stream(hours, seed=seed + 17 * s, ws_mean=10.0 + 12.0 * s,
                                               wd0=90.0 * s) for s in range(1, n_scen)]
    return w, np.stack([np.asarray(x, dtype=np.float64).reshape(hours, 4) for x in weathers])


def _load(ctx, w, weathers, probs):
    L = w.landscape
    lid = ctx.load_landscape(L.fuel, L.slope, L.aspect, L.unburnable, L.cell_size)
    ctx.set_weather_scenarios(lid, weathers, probs)
    return lid


def _oracle(w, weathers, probs):
    L = w.landscape
    return oracle.ScenarioOracle(L.fuel, L.slope, L.aspect, L.unburnable, L.cell_size,
                                 weathers=list(weathers), probs=probs, **w.params)


def _run(ctx, lid, w, **over):
    p = _params(**dict(w.params, **over))
    sid = ctx.simulate(lid, p)
    n = w.landscape.fuel.size
    scars, ign = ctx.get_scars(sid, p.n_replicas, n, ign_steps=bool(p.outputs & c2f.OUT_IGN_STEPS))
    work, nign, cell = ctx.get_counters(sid, p.n_replicas)
    scen = ctx.get_scenarios(sid, p.n_replicas)
    return sid, dict(scars=scars, ign=ign, work=work, n_ignited=nign, ign_cell=cell, scen=scen)


@pytest.fixture(scope="module")
def ctx():
    c2f.build()
    with c2f.Context(0) as c:
        yield c
        c.set_table_mode(True)


@pytest.mark.parametrize("eager", [True, False])
def test_every_replica_matches_the_oracle(ctx, eager):
    probs = [0.5, 0.2, 0.3]
    w, weathers = _world()
    ctx.set_table_mode(eager)
    lid = _load(ctx, w, weathers, probs)
    sid, got = _run(ctx, lid, w)
    so = _oracle(w, weathers, probs)
    R = w.params["n_replicas"]
    assert sorted(set(got["scen"].tolist())) == [0, 1, 2]
    for r in range(R):
        ref = so.run_replica(r)
        assert got["scen"][r] == ref["scenario"], r
        assert np.array_equal(got["ign"][r], ref["ign"].ravel()), r
        assert got["work"][r] == ref["work"], r
        assert got["n_ignited"][r] == ref["n_ignited"], r
        assert got["ign_cell"][r] == ref["ignition_cell"], r
    counts = ctx.burn_prob(sid, w.landscape.fuel.size)
    assert np.array_equal(counts, oracle.burn_prob(got["scars"]))
    total = np.zeros_like(counts)
    for sc in range(3):   # per-scenario maps: the oracle's scars of the replicas that drew sc
        per = ctx.burn_prob_scenario(sid, sc, w.landscape.fuel.size)
        ref = oracle.burn_prob(np.stack([so.run_replica(r)["scar"].ravel() for r in range(R)
                                         if so.scenario(r) == sc]))
        assert np.array_equal(per, ref), sc
        total += per
    assert np.array_equal(total, counts)
    with pytest.raises(c2f.C2FError) as e:
        ctx.burn_prob_scenario(sid, 3, w.landscape.fuel.size)
    assert e.value.code == c2f.C2F_EINVAL
    so.close()
    ctx.release(lid)


def test_stacked_table_rows_match_the_oracle(ctx):
    probs = [1.0, 1.0, 2.0]
    w, weathers = _world(side=48, hours=3)
    ctx.set_table_mode(True)
    lid = _load(ctx, w, weathers, probs)
    so = _oracle(w, weathers, probs)
    p = _params(**w.params)
    n = w.landscape.fuel.size
    fuel = w.landscape.fuel.ravel()
    for s in range(3):
        for h in range(3):
            _, hros, base = ctx.get_ros(lid, p, h, n, scenario=s)
            for cell in range(0, n, 5):
                if fuel[cell] == 0:
                    continue
                b, hr = so.base_inc(s, cell, h)
                assert np.array_equal(base[cell], b), (s, h, cell)
                assert hros[cell] == hr, (s, h, cell)
    with pytest.raises(c2f.C2FError) as e:
        ctx.get_ros(lid, p, 0, n, scenario=3)
    assert e.value.code == c2f.C2F_EINVAL
    so.close()
    ctx.release(lid)


def test_one_hot_equals_the_single_stream_run(ctx):
    w, weathers = _world(seed=32)
    ctx.set_table_mode(True)
    lid = _load(ctx, w, weathers, [0.0, 0.0, 1.0])
    _, got = _run(ctx, lid, w)
    assert (got["scen"] == 2).all()
    L = w.landscape
    lid1 = ctx.load_landscape(L.fuel, L.slope, L.aspect, L.unburnable, L.cell_size)
    ctx.set_weather(lid1, weathers[2])
    _, ref = _run(ctx, lid1, w)
    for k in ("scars", "ign", "work", "n_ignited", "ign_cell"):
        assert np.array_equal(got[k], ref[k]), k
    assert (ref["scen"] == 0).all()
    ctx.release(lid)
    ctx.release(lid1)


def test_batch_and_serving_equal_plain_runs(ctx):
    """A scenario landscape and a single-stream landscape in one batch and in
    one served epoch: every output equals its plain run."""
    w1, we1 = _world(side=60, n_replicas=30, seed=33)
    w2 = S.config2(side=45, n_replicas=20, hours=3)
    ctx.set_table_mode(True)
    lid1 = _load(ctx, w1, we1, [0.3, 0.3, 0.4])
    L2 = w2.landscape
    lid2 = ctx.load_landscape(L2.fuel, L2.slope, L2.aspect, L2.unburnable, L2.cell_size)
    ctx.set_weather(lid2, w2.weather)
    _, a1 = _run(ctx, lid1, w1)
    _, a2 = _run(ctx, lid2, w2)
    p1, p2 = _params(**w1.params), _params(**w2.params)
    s1, s2 = ctx.simulate_batch([lid1, lid2], [p1, p2])
    n1, n2 = w1.landscape.fuel.size, L2.fuel.size
    assert np.array_equal(ctx.get_scars(s1, p1.n_replicas, n1, ign_steps=True)[1], a1["ign"])
    assert np.array_equal(ctx.get_scenarios(s1, p1.n_replicas), a1["scen"])
    assert np.array_equal(ctx.get_scars(s2, p2.n_replicas, n2, ign_steps=True)[1], a2["ign"])
    ctx.set_serving(max_inflight=2, max_epoch_replicas=1 << 16, hbm_reserve_bytes=0)
    q1, q2 = ctx.submit(lid1, p1), ctx.submit(lid2, p2)
    ctx.wait(q1)
    ctx.wait(q2)
    assert np.array_equal(ctx.get_scars(q1, p1.n_replicas, n1, ign_steps=True)[1], a1["ign"])
    assert np.array_equal(ctx.get_scenarios(q1, p1.n_replicas), a1["scen"])
    assert np.array_equal(ctx.get_counters(q2, p2.n_replicas)[0], a2["work"])
    ctx.release(lid1)
    ctx.release(lid2)


def test_scenario_frequencies_at_scale(ctx):
    """20,000 replicas, 4 scenarios, one of probability 0: the drawn scenarios
    are the oracle's for every replica (an integer decision, bit-exact)."""
    probs = [0.1, 0.0, 0.3, 0.6]
    w, weathers = _world(side=40, n_replicas=20000, hours=1, n_scen=4, seed=34)
    ctx.set_table_mode(True)
    lid = _load(ctx, w, weathers, probs)
    _, got = _run(ctx, lid, w, outputs=c2f.OUT_SCARS | c2f.OUT_COUNTERS)
    thr = oracle.scenario_thresholds(probs)
    ref = np.array([oracle.scenario_of(w.params["seed"], r, thr) for r in range(20000)])
    assert np.array_equal(got["scen"], ref)
    assert (got["scen"] != 1).all()
    ctx.release(lid)


def test_bad_scenario_inputs_are_rejected(ctx):
    w, weathers = _world(side=20, hours=2)
    L = w.landscape
    lid = ctx.load_landscape(L.fuel, L.slope, L.aspect, L.unburnable, L.cell_size)
    for probs in ([0.0, 0.0, 0.0], [1.0, -1.0, 1.0], [1.0, float("nan"), 1.0]):
        with pytest.raises(c2f.C2FError) as e:
            ctx.set_weather_scenarios(lid, weathers, probs)
        assert e.value.code == c2f.C2F_EINVAL
    big = np.repeat(weathers[:1, :1], 30000, axis=1)   # 3 x 30000 hours > 65535 rows
    with pytest.raises(c2f.C2FError) as e:
        ctx.set_weather_scenarios(lid, np.repeat(big, 3, axis=0), [1, 1, 1])
    assert e.value.code == c2f.C2F_EINVAL
    ctx.release(lid)


def test_full_size_scenarios_sampled():
    """The scenario workload as the benchmark runs it: 512 x 512, 8 streams of
    24 h, 1000 replicas; every replica's drawn scenario and a sample of
    replicas (the first and last of two scenarios) replayed by the oracle."""
    c2f.build()
    w = S.config2()
    weathers, probs = S.scenario_set(8, 24)
    with c2f.Context(0) as ctx:
        lid = _load(ctx, w, weathers, probs)
        p = _params(**dict(w.params, outputs=c2f.OUT_SCARS | c2f.OUT_COUNTERS))
        sid = ctx.simulate(lid, p)
        scen = ctx.get_scenarios(sid, 1000)
        work, nign, cell = ctx.get_counters(sid, 1000)
        thr = oracle.scenario_thresholds(probs)
        assert np.array_equal(scen, [oracle.scenario_of(w.params["seed"], r, thr) for r in range(1000)])
        so = _oracle(w, weathers, probs)
        picks = []
        for s_ in (0, 7):
            idx = np.flatnonzero(scen == s_)
            picks += [int(idx[0]), int(idx[-1])]
        for r in picks:
            ref = so.run_replica(r)
            scar, _ = ctx.get_replica_scar(sid, r, w.landscape.fuel.size)
            assert ref["scenario"] == scen[r]
            assert np.array_equal(scar, ref["scar"].ravel()), r
            assert work[r] == ref["work"] and nign[r] == ref["n_ignited"] and cell[r] == ref["ignition_cell"], r
        so.close()


def test_scenarios_with_burning_hours(ctx):
    """Weather scenarios and a drawn burning-hours limit together: every replica
    equals the oracle (each draw has its own Philox counter)."""
    probs = [0.4, 0.6]
    w, weathers = _world(side=50, n_replicas=24, hours=30, n_scen=2, seed=35)
    over = dict(burn_hours_min=2, burn_hours_max=9)
    w.params.update(over)
    ctx.set_table_mode(True)
    lid = _load(ctx, w, weathers, probs)
    _, got = _run(ctx, lid, w)
    so = _oracle(w, weathers, probs)
    for r in range(24):
        ref = so.run_replica(r)
        assert got["scen"][r] == ref["scenario"], r
        assert np.array_equal(got["ign"][r], ref["ign"].ravel()), r
        assert got["work"][r] == ref["work"], r
    so.close()
    ctx.release(lid)


def test_single_scenario_and_null_probabilities(ctx):
    """One scenario through the scenario call (probabilities may be NULL) is the
    plain single-stream run; zero-weight scenarios are never drawn."""
    w, weathers = _world(side=30, n_replicas=12, hours=2, seed=36)
    L = w.landscape
    ctx.set_table_mode(True)
    lid = ctx.load_landscape(L.fuel, L.slope, L.aspect, L.unburnable, L.cell_size)
    one = np.ascontiguousarray(weathers[:1], dtype=np.float64)
    ctx._check(ctx.lib.c2f_set_weather_scenarios(ctx.h, lid, 1, one.shape[1],
                                                  one.ctypes.data_as(c2f.C.c_void_p), None))
    _, a = _run(ctx, lid, w)
    ctx.set_weather(lid, weathers[0])
    _, b = _run(ctx, lid, w)
    for k in ("ign", "work", "n_ignited", "ign_cell"):
        assert np.array_equal(a[k], b[k]), k
    assert (a["scen"] == 0).all()
    with pytest.raises(c2f.C2FError) as e:      # several scenarios need probabilities
        ctx._check(ctx.lib.c2f_set_weather_scenarios(ctx.h, lid, 3, weathers.shape[1],
                                                      np.ascontiguousarray(weathers).ctypes.data_as(c2f.C.c_void_p),
                                                      None))
    assert e.value.code == c2f.C2F_EINVAL
    ctx.release(lid)
