"""Serving (asynchronous submit / poll / wait / cancel with continuous batching).

A request's results must not depend on what else is being served: the scars,
work counts and ignition counts of a simulation submitted in a mix of other
requests (several landscapes, epochs overlapping on the device, requests
joining later epochs) equal those of the same simulation run alone with
c2f_simulate, bit for bit.  Each replica's random numbers are keyed by
(seed, replica, cell, hour) only (Sec. 3.4 replicas are independent), so this
is exact equality.
"""
import numpy as np
import pytest

import c2f_synth as S
import paper_1905_09317_gb300 as c2f

pytestmark = pytest.mark.gpu

_KEYS = {f[0] for f in c2f.SimParams._fields_}


def _params(**kw):
    return c2f.default_params(**{k: v for k, v in kw.items() if k in _KEYS})


def _landscapes(ctx):
    out = []
    for i, side in enumerate((64, 97, 130)):
        L = S.heterogeneous_landscape(side, side, seed=100 + i)
        lid = ctx.load_landscape(L.fuel, L.slope, L.aspect, cell_size=L.cell_size)
        ctx.set_weather(lid, S.weather_stream(12, seed=200 + i))
        out.append((lid, L.fuel.size))
    return out


def _requests(lands, n=14, seed=5):
    rng = np.random.default_rng(seed)
    reqs = []
    for q in range(n):
        lid, n_cells = lands[q % len(lands)]
        p = _params(seed=1000 + q, n_replicas=int(rng.integers(1, 40)), hours=int(rng.integers(1, 7)),
                    ignition_mode=1, ros_sigma=0.1 * (q % 3), burnout_delta=float(q % 2))
        reqs.append((lid, n_cells, p))
    return reqs


def _results(ctx, sid, p, n_cells):
    scars, _ = ctx.get_scars(sid, p.n_replicas, n_cells)
    work, nign, cell = ctx.get_counters(sid, p.n_replicas)
    return scars, work, nign, cell


def _same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


def test_request_alone_equals_request_in_a_mix():
    c2f.build()
    with c2f.Context(0) as ctx:
        lands = _landscapes(ctx)
        reqs = _requests(lands)
        alone = []
        for lid, n_cells, p in reqs:
            sid = ctx.simulate(lid, p)
            alone.append(_results(ctx, sid, p, n_cells))
            ctx.release(sid)
        # several small epochs, two in flight: later requests join later epochs
        ctx.set_serving(max_inflight=2, max_epoch_replicas=60, hbm_reserve_bytes=0)
        sids = [ctx.submit(lid, p) for lid, _, p in reqs]
        pending = set(sids)
        for _ in range(200000):
            pending = {s for s in pending if not ctx.poll(s)}
            if not pending:
                break
        else:
            raise AssertionError("served requests did not finish")
        for sid, (lid, n_cells, p), ref in zip(sids, reqs, alone):
            assert _same(_results(ctx, sid, p, n_cells), ref), sid


def test_wait_and_interleaved_submits():
    c2f.build()
    with c2f.Context(0) as ctx:
        lands = _landscapes(ctx)
        reqs = _requests(lands, n=9, seed=11)
        alone = []
        for lid, n_cells, p in reqs:
            sid = ctx.simulate(lid, p)
            alone.append(_results(ctx, sid, p, n_cells))
        ctx.set_serving(max_inflight=3, max_epoch_replicas=1 << 16, hbm_reserve_bytes=0)
        got = {}
        sids = []
        for i, (lid, n_cells, p) in enumerate(reqs):
            sids.append(ctx.submit(lid, p))
            if i % 3 == 2:   # a client that reads an earlier answer while submitting more
                j = i - 2
                ctx.wait(sids[j])
                got[j] = _results(ctx, sids[j], reqs[j][2], reqs[j][1])
        for j, sid in enumerate(sids):
            ctx.wait(sid)
            got.setdefault(j, _results(ctx, sid, reqs[j][2], reqs[j][1]))
        for j in range(len(reqs)):
            assert _same(got[j], alone[j]), j


def test_queued_request_is_busy_then_cancel():
    c2f.build()
    with c2f.Context(0) as ctx:
        lands = _landscapes(ctx)
        lid, n_cells = lands[2]
        ctx.set_serving(max_inflight=1, max_epoch_replicas=64, hbm_reserve_bytes=0)
        big = _params(seed=3, n_replicas=64, hours=6, ignition_mode=1)
        s1 = ctx.submit(lid, big)
        s2 = ctx.submit(lid, _params(seed=4, n_replicas=8, hours=3, ignition_mode=1))
        s3 = ctx.submit(lid, _params(seed=5, n_replicas=8, hours=3, ignition_mode=1))
        # one epoch in flight at most: s2 and s3 wait in the queue, and reading
        # a result does not advance the scheduler
        with pytest.raises(c2f.C2FError) as e:
            ctx.get_counters(s2, 8)
        assert e.value.code == c2f.C2F_EBUSY
        ctx.cancel(s2)
        with pytest.raises(c2f.C2FError) as e:
            ctx.wait(s2)
        assert e.value.code == c2f.C2F_ECANCELED
        with pytest.raises(c2f.C2FError) as e:
            ctx.get_scars(s2, 8, n_cells)
        assert e.value.code == c2f.C2F_ECANCELED
        ctx.wait(s3)
        ctx.wait(s1)
        ref = ctx.simulate(lid, _params(seed=5, n_replicas=8, hours=3, ignition_mode=1))
        assert _same(_results(ctx, s3, _params(n_replicas=8), n_cells),
                     _results(ctx, ref, _params(n_replicas=8), n_cells))


def test_release_while_queued_and_weather_change_while_running():
    c2f.build()
    with c2f.Context(0) as ctx:
        lands = _landscapes(ctx)
        lid, n_cells = lands[1]
        p = _params(seed=8, n_replicas=24, hours=5, ignition_mode=1, ros_sigma=0.2)
        ref = _results(ctx, ctx.simulate(lid, p), p, n_cells)
        ctx.set_serving(max_inflight=1, max_epoch_replicas=24, hbm_reserve_bytes=0)
        s1 = ctx.submit(lid, p)
        s2 = ctx.submit(lid, p)
        ctx.release(s2)               # dropped from the queue
        # new weather: s1 keeps the table it was submitted with
        ctx.set_weather(lid, S.weather_stream(12, seed=999))
        ctx.wait(s1)
        assert _same(_results(ctx, s1, p, n_cells), ref)
        with pytest.raises(c2f.C2FError) as e:
            ctx.wait(s2)
        assert e.value.code == c2f.C2F_ENOTFOUND
