"""Burning hours per day on the GPU vs the oracle (needs a GB300).

A5, general fire dynamics condition (1): a replica's fire burns only in the
weather hours h with h mod 24 < B, B constant or drawn per replica from
{min..max}; in the other hours it is dormant.  Every replica is compared bit
for bit with the oracle (ignition steps, work, ignited count), with eager and
on-demand tables, with coarse fire periods, and in a batch.
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


def _world(side=60, R=20, hours=52, seed=41):
    w = S.config2(side=side, n_replicas=R, hours=hours)
    w.weather = S.weather_stream(hours, seed=seed, ws_mean=14.0)
    w.params["seed"] = seed
    return w


@pytest.fixture(scope="module")
def ctx():
    c2f.build()
    with c2f.Context(0) as c:
        yield c
        c.set_table_mode(True)


def _gpu(ctx, w, **over):
    L = w.landscape
    lid = ctx.load_landscape(L.fuel, L.slope, L.aspect, L.unburnable, L.cell_size)
    ctx.set_weather(lid, w.weather)
    p = _params(**dict(w.params, **over))
    sid = ctx.simulate(lid, p)
    _, ign = ctx.get_scars(sid, p.n_replicas, L.fuel.size, ign_steps=True)
    work, nign, cell = ctx.get_counters(sid, p.n_replicas)
    ctx.release(lid)
    return dict(ign=ign, work=work, n_ignited=nign, ign_cell=cell)


def _check_all(w, got, **over):
    L = w.landscape
    o = oracle.Oracle(L.fuel, L.slope, L.aspect, L.unburnable, cell_size=L.cell_size,
                      weather=w.weather, **dict(w.params, **over))
    for r in range(w.params["n_replicas"]):
        ref = o.run_replica(r)
        assert np.array_equal(got["ign"][r], ref["ign"].ravel()), r
        assert got["work"][r] == ref["work"], r
        assert got["n_ignited"][r] == ref["n_ignited"], r
    o.close()


@pytest.mark.parametrize("eager", [True, False])
def test_drawn_burning_hours_match_the_oracle(ctx, eager):
    w = _world()
    ctx.set_table_mode(eager)
    over = dict(burn_hours_min=3, burn_hours_max=10)
    _check_all(w, _gpu(ctx, w, **over), **over)


@pytest.mark.parametrize("over", [dict(burn_hours_min=4, burn_hours_max=4, minutes_per_step=10),
                                  dict(burn_hours_min=1, burn_hours_max=2, burnout_delta=1.0),
                                  dict(burn_hours_min=6, burn_hours_max=6, ros_threshold=2.0)])
def test_constant_and_options(ctx, over):
    w = _world(side=48, R=12, hours=50, seed=42)
    ctx.set_table_mode(True)
    _check_all(w, _gpu(ctx, w, **over), **over)


def test_24_hours_equals_no_limit(ctx):
    w = _world(side=50, R=10, hours=30, seed=43)
    ctx.set_table_mode(True)
    a = _gpu(ctx, w)
    b = _gpu(ctx, w, burn_hours_min=24, burn_hours_max=24)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_batch_equals_plain_and_bad_values(ctx):
    w = _world(side=44, R=9, hours=30, seed=44)
    L = w.landscape
    ctx.set_table_mode(True)
    lid = ctx.load_landscape(L.fuel, L.slope, L.aspect, L.unburnable, L.cell_size)
    ctx.set_weather(lid, w.weather)
    p1 = _params(**dict(w.params, burn_hours_min=2, burn_hours_max=7))
    p2 = _params(**dict(w.params, seed=45))
    plain = [ctx.get_scars(ctx.simulate(lid, p), p.n_replicas, L.fuel.size, ign_steps=True)[1] for p in (p1, p2)]
    sids = ctx.simulate_batch([lid, lid], [p1, p2])
    for sid, p, ref in zip(sids, (p1, p2), plain):
        assert np.array_equal(ctx.get_scars(sid, p.n_replicas, L.fuel.size, ign_steps=True)[1], ref)
    for lo, hi in ((0, 5), (5, 4), (1, 25), (-1, 3)):
        with pytest.raises(c2f.C2FError) as e:
            ctx.simulate(lid, _params(**dict(w.params, burn_hours_min=lo, burn_hours_max=hi)))
        assert e.value.code == c2f.C2F_EINVAL
    ctx.release(lid)
