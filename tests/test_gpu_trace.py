"""Launch trace (c2f_trace) of the table build and the frontier (needs a GPU).

Checked against what the launches fix: one record per K1 CTA (grid of
ceil(cells / 128) x hours, each hour as often as there are column blocks)
and one per replica, the table's records all ending before the frontier
that reads it starts (same stream), SM ids below the SM count, starts before
ends, nothing written past the capacity (records beyond it are counted),
and results bit-identical with tracing on or off.
"""
import ctypes as C

import numpy as np
import pytest

import c2f_synth as S
import paper_1905_09317_gb300 as c2f

pytestmark = pytest.mark.gpu


def _params(w):
    keys = {f[0] for f in c2f.SimParams._fields_}
    return c2f.default_params(**{k: v for k, v in w.params.items() if k in keys})


def _records(buf, n):
    rec = buf.view(-1, 4)[:n].cpu().numpy().view(np.uint64)
    return (rec[:, 0] & 0xFF).astype(np.int64), ((rec[:, 0] >> 8) & 0xFFFFFF).astype(np.int64), \
        (rec[:, 0] >> 32).astype(np.int64), rec[:, 1].astype(np.int64), rec[:, 2].astype(np.int64), \
        rec[:, 3].astype(np.int64)


def test_trace_records_every_table_cta_and_replica():
    torch = pytest.importorskip("torch")
    c2f.build()
    w = S.config2(side=160, n_replicas=40, hours=3)
    L = w.landscape
    n = L.fuel.size
    p = _params(w)
    R, H = p.n_replicas, p.hours
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    with c2f.Context(0) as ctx:
        lid = ctx.load_landscape(L.fuel, L.slope, L.aspect, cell_size=L.cell_size)
        ctx.set_weather(lid, w.weather)
        sid = ctx.simulate(lid, p)
        ref = (ctx.get_scars(sid, R, n)[0],) + tuple(ctx.get_counters(sid, R))
        ctx.release(sid)

        cap = 50_000
        guard = 64
        buf = torch.full(((cap + guard) * 4,), -1, dtype=torch.int64, device="cuda")
        ctx.trace(buf.data_ptr(), cap)
        assert ctx.trace_count() == 0
        ctx.build_ros(lid, p, force=1)
        sid = ctx.simulate(lid, p)
        got = (ctx.get_scars(sid, R, n)[0],) + tuple(ctx.get_counters(sid, R))
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)
        cnt = ctx.trace_count()
        blocks = -(-n // 128)
        assert cnt == blocks * H + R
        kind, sm, aux, tag, t0, t1 = _records(buf, cnt)
        assert np.all(buf.view(-1, 4)[cnt:].cpu().numpy() == -1)        # nothing past the records
        assert np.all(t1 >= t0) and np.all(sm < sms)
        tab, rep = kind == c2f.TRACE_TABLE, kind == c2f.TRACE_REPLICA
        assert tab.sum() == blocks * H and rep.sum() == R
        assert np.array_equal(np.bincount(aux[tab], minlength=H), np.full(H, blocks))
        assert np.array_equal(np.sort(aux[rep]), np.arange(R))
        assert np.unique(tag[tab]).size == 1 and np.unique(tag[rep]).size == 1
        # the frontier reads the table: it starts after the build's last CTA ends
        # (the global timer ticks in steps of up to a microsecond)
        assert t1[tab].max() <= t0[rep].min() + 2000
        ctx.release(sid)

        # a second simulation gets the next creation number
        sid = ctx.simulate(lid, p)
        cnt2 = ctx.trace_count()
        assert cnt2 == cnt + R
        kind2, _, _, tag2, _, _ = _records(buf, cnt2)
        assert np.unique(tag2[cnt:]).size == 1 and tag2[cnt] == tag[rep][0] + 1
        ctx.release(sid)

        # a capacity smaller than the work: the excess is counted, not written
        buf[:] = -1
        ctx.trace(buf.data_ptr(), 10)
        sid = ctx.simulate(lid, p)
        assert ctx.trace_count() == R
        host = buf.view(-1, 4).cpu().numpy()
        assert np.all(host[:10, 2] >= 0) and np.all(host[10:] == -1)
        ctx.release(sid)

        # off: the count stays; bad arguments are refused
        ctx.trace(None)
        before = ctx.trace_count()
        ctx.release(ctx.simulate(lid, p))
        assert ctx.trace_count() == before
        assert ctx.lib.c2f_trace(ctx.h, C.c_void_p(buf.data_ptr()), 0) == c2f.C2F_EINVAL
        assert ctx.lib.c2f_trace(ctx.h, None, 5) == c2f.C2F_EINVAL


def test_trace_covers_batched_and_served_simulations():
    """A batch of two landscapes (one CUDA graph) and two served requests: every
    table build and every replica is recorded once, one tag per simulation."""
    torch = pytest.importorskip("torch")
    c2f.build()
    wa = S.config2(side=96, n_replicas=24, hours=2)
    wb = S.config2(side=130, n_replicas=16, hours=3)
    pa, pb = _params(wa), _params(wb)
    with c2f.Context(0) as ctx:
        lids = []
        for w in (wa, wb):
            L = w.landscape
            lid = ctx.load_landscape(L.fuel, L.slope, L.aspect, cell_size=L.cell_size)
            ctx.set_weather(lid, w.weather)
            lids.append(lid)
        cap = 20_000
        buf = torch.full((cap * 4,), -1, dtype=torch.int64, device="cuda")
        ctx.trace(buf.data_ptr(), cap)
        sids = ctx.simulate_batch(lids, [pa, pb])
        cnt = ctx.trace_count()
        na, nb = wa.landscape.fuel.size, wb.landscape.fuel.size
        blocks = (-(-na // 128)) * pa.hours + (-(-nb // 128)) * pb.hours
        assert cnt == blocks + pa.n_replicas + pb.n_replicas
        kind, _, aux, tag, t0, t1 = _records(buf, cnt)
        rep = kind == c2f.TRACE_REPLICA
        tags = np.unique(tag[rep])
        assert tags.size == 2
        assert sorted(np.bincount(np.searchsorted(tags, tag[rep]))) == sorted([pa.n_replicas, pb.n_replicas])
        assert np.unique(tag[kind == c2f.TRACE_TABLE]).size == 2 and np.all(t1 >= t0)
        for s in sids:
            ctx.release(s)

        # served: the tables are built, so only replicas are recorded
        ctx.trace(buf.data_ptr(), cap)
        ctx.set_serving(max_inflight=2)
        s1, s2 = ctx.submit(lids[0], pa), ctx.submit(lids[1], pb)
        ctx.wait(s1)
        ctx.wait(s2)
        cnt = ctx.trace_count()
        assert cnt == pa.n_replicas + pb.n_replicas
        kind, _, aux, tag, _, _ = _records(buf, cnt)
        assert np.all(kind == c2f.TRACE_REPLICA) and np.unique(tag).size == 2
        ctx.trace(None)
        ctx.release(s1)
        ctx.release(s2)
