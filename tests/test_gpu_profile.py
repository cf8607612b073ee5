"""Per-replica frontier counters and kernel timing (needs a GPU).

The counters (c2f_get_replica_profile) are a measuring instrument, so they are
checked against what the run itself fixes: every period in which a cell
ignited was visited, the cells ignited after period 0 are the ignited count
minus the ignition cell, a round holds 1..32 crossing cells and a new-cell
pass 1..4 cells, phase cycles add up to at most the total.  Switching them on
must not change a single result bit, and compactions forced by a small list
capacity show up in their own counter.
"""
import numpy as np
import pytest

import c2f_synth as S
import paper_1905_09317_gb300 as c2f

pytestmark = pytest.mark.gpu


def _run(ctx, lid, p, n):
    sid = ctx.simulate(lid, p)
    scars, ign = ctx.get_scars(sid, p.n_replicas, n, ign_steps=True)
    work, nign, cell = ctx.get_counters(sid, p.n_replicas)
    return sid, (scars, ign, work, nign, cell)


def _check_counters(pr, ign, nign, H, sph):
    assert pr.shape[1] == 16
    total, bound, send, new, periods, hits, newc, longest, walk, comp, rounds, newit = pr[:, :12].T
    assert np.all(pr[:, 12:] == 0)
    assert np.array_equal(newc, nign.astype(np.int64) - 1)            # every ignition after period 0
    for r in range(pr.shape[0]):
        steps = np.unique(ign[r][ign[r] > 0])
        assert periods[r] >= steps.size, r                            # each ignition period was visited
    assert np.all(periods <= H * sph)
    assert np.all(total >= bound + send + new) and np.all(total > 0)
    assert np.all(walk <= send)
    assert np.all((rounds <= hits) & (hits <= 32 * rounds))
    assert np.all((newit <= newc) & (newc <= 4 * newit))
    assert np.all(longest[periods > 0] >= 1)


def test_replica_counters_consistent_and_harmless():
    c2f.build()
    w = S.config2(side=200, n_replicas=48, hours=12)
    L = w.landscape
    n = L.fuel.size
    keys = {f[0] for f in c2f.SimParams._fields_}
    p = c2f.default_params(**{k: v for k, v in w.params.items() if k in keys})
    p.outputs = c2f.OUT_SCARS | c2f.OUT_IGN_STEPS | c2f.OUT_COUNTERS
    sph = 60 // p.minutes_per_step
    with c2f.Context(0) as ctx:
        lid = ctx.load_landscape(L.fuel, L.slope, L.aspect, cell_size=L.cell_size)
        ctx.set_weather(lid, w.weather)
        sid, ref = _run(ctx, lid, p, n)
        with pytest.raises(c2f.C2FError) as e:                       # run without the counters
            ctx.replica_profile(sid, p.n_replicas)
        assert e.value.code == c2f.C2F_EINVAL
        ctx.release(sid)

        # kernel timing alone: no counters, same results
        ctx.profile(True)
        ctx.kernel_times()
        sid, got = _run(ctx, lid, p, n)
        kt = ctx.kernel_times()
        assert kt["frontier"][1] >= 1 and kt["frontier"][0] > 0
        with pytest.raises(c2f.C2FError):
            ctx.replica_profile(sid, p.n_replicas)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)
        ctx.release(sid)

        # counters on
        ctx.profile(True, replicas=True)
        sid, got = _run(ctx, lid, p, n)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)
        pr = ctx.replica_profile(sid, p.n_replicas)
        _check_counters(pr, got[1], got[3], p.hours, sph)
        ctx.release(sid)

        # a small list capacity and an early compaction trigger: compactions
        # are counted, results unchanged
        ctx.set_list_capacity(128)
        ctx.set_compaction(2)
        sid, got = _run(ctx, lid, p, n)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)
        pr2 = ctx.replica_profile(sid, p.n_replicas)
        _check_counters(pr2, got[1], got[3], p.hours, sph)
        assert pr2[:, 9].sum() > 0
        ctx.release(sid)

        # only the two documented flags
        assert ctx.lib.c2f_profile(ctx.h, 4) == c2f.C2F_EINVAL
        ctx.profile(False)
