"""Eager vs on-demand rate-of-spread tables (needs a GB300).

A table is eager (every (cell, hour) row written by the table kernel before
the frontier runs) or lazy (rows written by the frontier warps themselves,
32 cells at a time, the first time a burning cell of that chunk needs them).
The rows are the same function of the same inputs (Sec. 3.7, Eqs. 1-4), so
every simulation output must be bit-identical in the two modes, and both must
equal the oracle.
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


def _run(ctx, w, eager, **over):
    p = dict(w.params)
    p.update(over)
    L = w.landscape
    ctx.set_table_mode(eager)
    lid = ctx.load_landscape(L.fuel, L.slope, L.aspect, L.unburnable, L.cell_size)
    ctx.set_weather(lid, w.weather)
    gp = _params(**p)
    sid = ctx.simulate(lid, gp)
    n = L.fuel.size
    scars, ign = ctx.get_scars(sid, gp.n_replicas, n, ign_steps=True)
    work, nign, cells = ctx.get_counters(sid, gp.n_replicas)
    ctx.release(sid)
    ctx.release(lid)
    return dict(scars=scars, ign=ign, work=work, n_ignited=nign, ign_cell=cells)


def _same(a, b):
    for k in a:
        assert np.array_equal(a[k], b[k]), k


@pytest.fixture(scope="module")
def ctx():
    c2f.build()
    with c2f.Context(0) as c:
        yield c
        c.set_table_mode(False)


@pytest.mark.parametrize("over", [dict(), dict(ellipse_mode=1), dict(ros_threshold=2.5),
                                  dict(burnout_delta=1.5), dict(minutes_per_step=10),
                                  dict(ros_sigma=0.0), dict(const_ros=12.0)])
def test_lazy_equals_eager(ctx, over):
    w = S.config2(side=75, n_replicas=40, hours=5)
    lazy = _run(ctx, w, False, **over)
    eager = _run(ctx, w, True, **over)
    _same(lazy, eager)


def test_lazy_beyond_the_window_matches_oracle(ctx):
    """A landscape wider and taller than the 256 x 256 shared-memory window:
    chunks outside it are tracked in device memory only."""
    w = S.config2(side=700, n_replicas=12, hours=10)
    w.params["seed"] = 4242
    lazy = _run(ctx, w, False)
    eager = _run(ctx, w, True)
    _same(lazy, eager)
    L = w.landscape
    o = oracle.Oracle(L.fuel, L.slope, L.aspect, L.unburnable, cell_size=L.cell_size,
                      weather=w.weather, **w.params)
    for r in (0, 5, 11):
        ref = o.run_replica(r)
        assert np.array_equal(lazy["ign"][r], ref["ign"].ravel()), r
        assert lazy["work"][r] == ref["work"], r


def test_exported_rows_after_a_lazy_run_match_the_oracle(ctx):
    """get_ros on a table that a lazy run filled in part: the table kernel
    completes it and every exported row is the oracle's."""
    w = S.config2(side=64, n_replicas=30, hours=3)
    L = w.landscape
    ctx.set_table_mode(False)
    lid = ctx.load_landscape(L.fuel, L.slope, L.aspect, L.unburnable, L.cell_size)
    ctx.set_weather(lid, w.weather)
    p = _params(**w.params)
    ctx.simulate(lid, p)
    o = oracle.Oracle(L.fuel, L.slope, L.aspect, L.unburnable, cell_size=L.cell_size,
                      weather=w.weather, **w.params)
    n = L.fuel.size
    for h in range(3):
        _, hros, base = ctx.get_ros(lid, p, h, n)
        for cell in range(0, n, 7):
            if L.fuel.ravel()[cell] == 0:
                continue
            b, hr = o.base_inc(cell, h)
            assert np.array_equal(base[cell], b), (h, cell)
            assert hros[cell] == hr, (h, cell)
    ctx.release(lid)


def test_lazy_table_is_reused_and_extended(ctx):
    """A second simulation on the same lazy table (more replicas, a different
    seed) sees rows the first one wrote and fills the rest; results equal a
    run on a fresh eager table."""
    w = S.config2(side=90, n_replicas=20, hours=4)
    L = w.landscape
    ctx.set_table_mode(False)
    lid = ctx.load_landscape(L.fuel, L.slope, L.aspect, L.unburnable, L.cell_size)
    ctx.set_weather(lid, w.weather)
    ctx.simulate(lid, _params(**w.params))
    p2 = dict(w.params, seed=99, n_replicas=50)
    sid = ctx.simulate(lid, _params(**p2))
    n = L.fuel.size
    scars, ign = ctx.get_scars(sid, 50, n, ign_steps=True)
    ctx.release(lid)
    w2 = S.config2(side=90, n_replicas=50, hours=4)
    w2.params["seed"] = 99
    eager = _run(ctx, w2, True)
    assert np.array_equal(ign, eager["ign"]) and np.array_equal(scars, eager["scars"])


def test_batch_with_lazy_tables(ctx):
    ws = [S.config2(side=s, n_replicas=r, hours=h) for s, r, h in ((50, 7, 3), (120, 25, 5), (33, 3, 2))]
    ctx.set_table_mode(False)
    lids = []
    for w in ws:
        L = w.landscape
        lid = ctx.load_landscape(L.fuel, L.slope, L.aspect, L.unburnable, L.cell_size)
        ctx.set_weather(lid, w.weather)
        lids.append(lid)
    ps = [_params(**w.params) for w in ws]
    sids = ctx.simulate_batch(lids, ps)
    for w, sid, p in zip(ws, sids, ps):
        n = w.landscape.fuel.size
        _, ign = ctx.get_scars(sid, p.n_replicas, n, ign_steps=True)
        eager = _run(ctx, w, True)
        assert np.array_equal(ign, eager["ign"])
    ctx.set_table_mode(False)
    for lid in lids:
        ctx.release(lid)
