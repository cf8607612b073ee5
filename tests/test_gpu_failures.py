"""Failure paths of the library, made on the host or by a bounded wait (needs a GPU).

No test here faults, traps or hangs the GPU:
- allocation failure: the context's allocation hooks refuse the k-th device
  allocation of a call; the call must return C2F_ENOMEM, leave its outputs
  untouched, and the context must stay usable (the next call gives the same
  results as a clean run);
- serving admission: with a device-memory reserve larger than the device,
  queued work is held back until the running epoch ends (an epoch is still
  admitted when nothing else runs), and results do not change;
- bounded wait: a lazy-table chunk is marked as being computed by a warp that
  never finishes; the frontier's wait for it gives up after the configured
  number of polls, the call returns C2F_ETIMEOUT and the context stays usable.
"""
import ctypes as C

import numpy as np
import pytest

import c2f_synth as S
import paper_1905_09317_gb300 as c2f

pytestmark = pytest.mark.gpu


def _small(side, n_replicas, hours, seed):
    """A config-2-style workload of another landscape and weather seed."""
    params = dict(seed=1000 + seed, n_replicas=n_replicas, hours=hours, minutes_per_step=1,
                  ignition_mode=1, ignition_cell=0, ros_sigma=0.1)
    return S.Workload(S.heterogeneous_landscape(side, seed=seed), S.weather_stream(hours, seed=100 + seed),
                      params)


def _params(w, **over):
    d = dict(w.params)
    d.update(over)
    keys = {f[0] for f in c2f.SimParams._fields_}
    return c2f.default_params(**{k: v for k, v in d.items() if k in keys})


def _load(ctx, w):
    L = w.landscape
    lid = ctx.load_landscape(L.fuel, L.slope, L.aspect, cell_size=L.cell_size)
    ctx.set_weather(lid, w.weather)
    return lid


def _results(ctx, sid, R, n):
    scars, _ = ctx.get_scars(sid, R, n)
    work, nign, cells = ctx.get_counters(sid, R)
    return scars, work, nign, cells, ctx.burn_prob(sid, n)


class FailingHooks:
    """Device memory from PyTorch's caching allocator; the `fail_at`-th
    allocation counted from the last reset is refused (returns NULL)."""

    def __init__(self, device):
        import torch
        self.fail_at = None
        self.count = 0

        def alloc(nbytes, stream, user):
            self.count += 1
            if self.fail_at is not None and self.count == self.fail_at:
                return None
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), device, int(stream or 0))
            except Exception:
                return None

        def free(ptr, nbytes, stream, user):
            torch.cuda.caching_allocator_delete(int(ptr))

        self.hooks = c2f.AllocHooks(c2f._ALLOC_FN(alloc), c2f._FREE_FN(free), None)

    def arm(self, k):
        self.count, self.fail_at = 0, k

    def disarm(self):
        self.fail_at = None


def test_allocation_failure_gives_enomem_and_a_usable_context():
    pytest.importorskip("torch")
    c2f.build()
    w = S.config2(side=80, n_replicas=24, hours=3)
    n = w.landscape.fuel.size
    p = _params(w)
    hooks = FailingHooks(0)
    with c2f.Context(0, allocator=hooks.hooks) as ctx:
        lid = _load(ctx, w)
        sid = ctx.simulate(lid, p)
        ref = _results(ctx, sid, p.n_replicas, n)
        ctx.release(sid)
        # refuse each allocation of a simulate in turn (the table is rebuilt
        # every time: set_weather drops it), until a call needs fewer
        failures = 0
        for k in range(1, 200):
            ctx.set_weather(lid, w.weather)
            out = C.c_int32(-12345)
            hooks.arm(k)
            rc = ctx.lib.c2f_simulate(ctx.h, lid, C.byref(p), C.byref(out))
            hooks.disarm()
            if hooks.count < k:            # the call made fewer than k allocations
                assert rc == c2f.C2F_OK
                got = _results(ctx, out.value, p.n_replicas, n)
                for a, b in zip(got, ref):
                    assert np.array_equal(a, b)
                ctx.release(out.value)
                break
            assert rc == c2f.C2F_ENOMEM, (k, rc)
            assert out.value == -12345, k          # no simulation id on failure
            failures += 1
            # the context is still usable: a clean call right after the failure
            if k % 4 == 1:
                sid = ctx.simulate(lid, p)
                got = _results(ctx, sid, p.n_replicas, n)
                for a, b in zip(got, ref):
                    assert np.array_equal(a, b), k
                ctx.release(sid)
        assert failures >= 5
        # an output call whose temporary allocation fails leaves the host buffer untouched
        sid = ctx.simulate(lid, p)
        counts = np.full(n, 0xDEADBEEF, dtype=np.uint32)
        hooks.arm(1)
        rc = ctx.lib.c2f_burn_prob(ctx.h, sid, C.c_void_p(counts.ctypes.data))
        hooks.disarm()
        assert rc == c2f.C2F_ENOMEM and np.all(counts == 0xDEADBEEF)
        assert np.array_equal(ctx.burn_prob(sid, n), ref[4])
        ctx.release(sid)
        # a batch whose allocations fail part-way through (graph path) leaves no
        # half-built table behind
        w2 = _small(48, 8, 2, 7)
        lid2 = _load(ctx, w2)
        p2 = _params(w2)
        sids = ctx.simulate_batch([lid, lid2], [p, p2])
        ref2 = _results(ctx, sids[1], p2.n_replicas, w2.landscape.fuel.size)
        for s in sids:
            ctx.release(s)
        for k in (2, 5, 9, 14):
            ctx.set_weather(lid, w.weather)
            ctx.set_weather(lid2, w2.weather)
            ids = (C.c_int32 * 2)(lid, lid2)
            ps = (c2f.SimParams * 2)(p, p2)
            outs = (C.c_int32 * 2)(-1, -1)
            hooks.arm(k)
            rc = ctx.lib.c2f_simulate_batch(ctx.h, 2, ids, ps, outs)
            hooks.disarm()
            if hooks.count < k:
                assert rc == c2f.C2F_OK
                for s in outs:
                    ctx.release(s)
                continue
            assert rc == c2f.C2F_ENOMEM and list(outs) == [-1, -1], k
            sids = ctx.simulate_batch([lid, lid2], [p, p2])
            got = _results(ctx, sids[0], p.n_replicas, n)
            got2 = _results(ctx, sids[1], p2.n_replicas, w2.landscape.fuel.size)
            for a, b in zip(got, ref):
                assert np.array_equal(a, b), k
            for a, b in zip(got2, ref2):
                assert np.array_equal(a, b), k
            for s in sids:
                ctx.release(s)


def test_admission_waits_for_device_memory():
    c2f.build()
    wa = S.config2(n_replicas=1000)                    # the 512^2 workload: several ms of GPU work
    wb = _small(64, 16, 2, 11)
    pa, pb = _params(wa), _params(wb)
    na, nb = wa.landscape.fuel.size, wb.landscape.fuel.size
    with c2f.Context(0) as ctx:
        la, lb = _load(ctx, wa), _load(ctx, wb)
        ref_a = _results(ctx, ctx.simulate(la, pa), pa.n_replicas, na)
        ref_b = _results(ctx, ctx.simulate(lb, pb), pb.n_replicas, nb)
        import torch
        _, total = torch.cuda.mem_get_info(0)
        # a reserve beyond the whole device: B may start only when nothing else runs
        ctx.set_serving(max_inflight=4, max_epoch_replicas=1 << 16, hbm_reserve_bytes=2 * total)
        before = ctx.serving_stats()
        sa = ctx.submit(la, pa)
        sb = ctx.submit(lb, pb)
        mid = ctx.serving_stats()
        ctx.wait(sb)
        assert ctx.poll(sa)                 # B was admitted only after A's epoch had ended
        after = ctx.serving_stats()
        assert mid["admission_waits"] > before["admission_waits"]
        assert after["epochs"] == before["epochs"] + 2
        for got, ref in ((_results(ctx, sa, pa.n_replicas, na), ref_a), (_results(ctx, sb, pb.n_replicas, nb), ref_b)):
            for a, b in zip(got, ref):
                assert np.array_equal(a, b)
        ctx.release(sa)
        ctx.release(sb)
        # with no reserve both are admitted at once, and the results are the same
        ctx.set_serving(max_inflight=4, max_epoch_replicas=1 << 16, hbm_reserve_bytes=0)
        w0 = ctx.serving_stats()["admission_waits"]
        sa = ctx.submit(la, pa)
        sb = ctx.submit(lb, pb)
        assert ctx.serving_stats()["admission_waits"] == w0
        ctx.wait(sa)
        ctx.wait(sb)
        for got, ref in ((_results(ctx, sa, pa.n_replicas, na), ref_a), (_results(ctx, sb, pb.n_replicas, nb), ref_b)):
            for a, b in zip(got, ref):
                assert np.array_equal(a, b)


def test_bounded_wait_for_a_held_chunk_times_out():
    c2f.build()
    w = _small(70, 6, 2, 5)
    L = w.landscape
    n = L.fuel.size
    burnable = np.flatnonzero(L.fuel.ravel() != 0)
    cell = int(burnable[len(burnable) // 2])
    p = _params(w, ignition_mode=0, ignition_cell=cell)
    with c2f.Context(0) as ctx:
        lid = _load(ctx, w)
        ctx.set_table_mode(True)
        ref = _results(ctx, ctx.simulate(lid, p), p.n_replicas, n)
        ctx.set_table_mode(False)
        ctx.build_ros(lid, p, force=2)                  # a new lazy table
        ctx.test_hold_chunk(lid, hour=0, cell=cell)     # the ignition cell's chunk never completes
        ctx.set_wait_limit(4000)                        # about half a millisecond of polls
        with pytest.raises(c2f.C2FError) as e:
            ctx.simulate(lid, p)
        assert e.value.code == c2f.C2F_ETIMEOUT
        # the context is still usable: a fresh lazy table, the default limit
        ctx.set_wait_limit(0)
        ctx.build_ros(lid, p, force=2)
        sid = ctx.simulate(lid, p)
        got = _results(ctx, sid, p.n_replicas, n)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)
        # hooks on tables that are not lazy, and out-of-range indices, are refused
        ctx.build_ros(lid, p, force=1)
        with pytest.raises(c2f.C2FError) as e:
            ctx.test_hold_chunk(lid, hour=0, cell=cell)
        assert e.value.code == c2f.C2F_EINVAL
        with pytest.raises(c2f.C2FError):
            ctx.set_wait_limit(-1)
