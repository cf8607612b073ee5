"""Output forms and device-memory hooks (needs a GB300).

Sec. 3.6 outputs: burn grids (bytes and bit-packed), the fire-scar evolution
by weather hour, and the device memory of a context coming from PyTorch's
caching allocator instead of the library's own stream-ordered allocations.
"""
import threading

import numpy as np
import pytest

import c2f_synth as S
import oracle
import paper_1905_09317_gb300 as c2f

pytestmark = pytest.mark.gpu

_KEYS = {f[0] for f in c2f.SimParams._fields_}


def _params(**kw):
    kw.setdefault("outputs", c2f.OUT_SCARS | c2f.OUT_COUNTERS | c2f.OUT_IGN_STEPS)
    return c2f.default_params(**{k: v for k, v in kw.items() if k in _KEYS})


def _simulate(ctx, w):
    L = w.landscape
    lid = ctx.load_landscape(L.fuel, L.slope, L.aspect, L.unburnable, L.cell_size)
    ctx.set_weather(lid, w.weather)
    sid = ctx.simulate(lid, _params(**w.params))
    return lid, sid


def test_bit_packed_scars_and_hourly_scars():
    c2f.build()
    w = S.config2(side=77, n_replicas=9, hours=4)
    rows, cols = w.landscape.fuel.shape
    n = rows * cols
    with c2f.Context(0) as ctx:
        lid, sid = _simulate(ctx, w)
        scars, ign = ctx.get_scars(sid, 9, n, ign_steps=True)
        words = ctx.get_scar_bits(sid, 9, rows, cols)
        bits = (words[:, :, :, None] >> np.arange(32, dtype=np.uint32)) & 1
        bits = bits.reshape(9, rows, -1)
        assert np.array_equal(bits[:, :, :cols].reshape(9, n).astype(np.uint8), scars)
        assert not bits[:, :, cols:].any()          # padding bits are zero
        o = oracle.Oracle(w.landscape.fuel, w.landscape.slope, w.landscape.aspect,
                          cell_size=w.landscape.cell_size, weather=w.weather, **w.params)
        for h in range(4):
            at = ctx.get_scars_at_hour(sid, h, 9, n)
            for r in (0, 4, 8):
                ref = o.run_replica(r)["ign"].ravel()
                assert np.array_equal(at[r], ((ref >= 0) & (ref <= 60 * (h + 1))).astype(np.uint8)), (h, r)
        assert np.array_equal(ctx.get_scars_at_hour(sid, 3, 9, n), scars)
        with pytest.raises(c2f.C2FError) as e:
            ctx.get_scars_at_hour(sid, 4, 9, n)
        assert e.value.code == c2f.C2F_EINVAL
        s2 = ctx.simulate(lid, _params(**dict(w.params, outputs=c2f.OUT_SCARS | c2f.OUT_COUNTERS)))
        with pytest.raises(c2f.C2FError) as e:
            ctx.get_scars_at_hour(s2, 0, 9, n)
        assert e.value.code == c2f.C2F_EINVAL


def test_torch_allocator_hooks_give_the_same_results():
    torch = pytest.importorskip("torch")
    c2f.build()
    w = S.config2(side=120, n_replicas=30, hours=5)
    n = w.landscape.fuel.size
    with c2f.Context(0) as ref_ctx:
        _, sid = _simulate(ref_ctx, w)
        ref_scars, ref_ign = ref_ctx.get_scars(sid, 30, n, ign_steps=True)
        ref_work = ref_ctx.get_counters(sid, 30)[0]
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated(0)
    ctx = c2f.Context(0, allocator="torch")
    lid, sid = _simulate(ctx, w)
    held = torch.cuda.memory_allocated(0) - base
    # the landscape, the table (72 B per cell-hour) and the outputs live in torch's pool
    assert held >= n * 5 * 72
    scars, ign = ctx.get_scars(sid, 30, n, ign_steps=True)
    assert np.array_equal(scars, ref_scars) and np.array_equal(ign, ref_ign)
    assert np.array_equal(ctx.get_counters(sid, 30)[0], ref_work)
    # serving epochs allocate on their own streams through the same hooks
    ctx.set_serving(max_inflight=2, max_epoch_replicas=30, hbm_reserve_bytes=0)
    s2 = ctx.submit(lid, _params(**w.params))
    ctx.wait(s2)
    assert np.array_equal(ctx.get_scars(s2, 30, n)[0], ref_scars)
    ctx.close()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated(0) == base


def test_last_error_is_per_thread():
    c2f.build()
    with c2f.Context(0) as ctx:
        lib = c2f.load_library()
        msgs = {}

        def worker():
            try:
                ctx.simulate(999, _params())
            except c2f.C2FError as e:
                msgs["worker"] = str(e)
            msgs["worker_after"] = lib.c2f_last_error(ctx.h).decode()

        with pytest.raises(c2f.C2FError):
            ctx.load_landscape(np.full((3, 3), 99, np.uint8))
        mine = lib.c2f_last_error(ctx.h).decode()
        t = threading.Thread(target=worker)
        t.start()
        t.join()
        assert "unknown landscape" in msgs["worker_after"]
        assert lib.c2f_last_error(ctx.h).decode() == mine and "fuel code" in mine


def test_release_right_after_asynchronous_reads():
    """Burn counts into device memory on a caller stream, the simulation released
    at once, and new simulations (whose allocations may reuse the freed memory)
    submitted on the context's epoch streams while the counts are being read: every
    step's counts equal a clean run's.  The same with the scar comparison."""
    torch = pytest.importorskip("torch")
    c2f.build()
    w = S.config2(side=192, n_replicas=200, hours=6)
    L = w.landscape
    n = L.fuel.size
    p = _params(**w.params)
    with c2f.Context(0) as ctx:
        lid = ctx.load_landscape(L.fuel, L.slope, L.aspect, cell_size=L.cell_size)
        ctx.set_weather(lid, w.weather)
        sid = ctx.simulate(lid, p)
        ref = ctx.burn_prob(sid, n)
        ctx.release(sid)
        stream = torch.cuda.Stream()
        ctx.set_stream(stream.cuda_stream)
        ctx.set_serving(max_inflight=3, max_epoch_replicas=p.n_replicas, hbm_reserve_bytes=0)
        outs = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in range(12)]
        pending = [ctx.submit(lid, p)]
        for i in range(12):
            pending.append(ctx.submit(lid, p))          # more work, more allocations
            sid = pending.pop(0)
            ctx.wait(sid)
            ctx.burn_prob_device(sid, outs[i].data_ptr())
            ctx.release(sid)                             # K4 may still be reading its scars
        for sid in pending:
            ctx.wait(sid)
            ctx.release(sid)
        torch.cuda.synchronize()
        for i, o in enumerate(outs):
            assert np.array_equal(o.cpu().numpy().view(np.uint32), ref), i
        # the scar comparison into device memory, both simulations released at once
        a, b = ctx.submit(lid, p), ctx.submit(lid, p)
        ctx.wait(a)
        ctx.wait(b)
        dn = torch.full((p.n_replicas,), -1.0, dtype=torch.float64, device="cuda")
        ctx.compare_scars_device(a, b, 0, 0, dn.data_ptr())
        ctx.release(a)
        ctx.release(b)
        c = ctx.submit(lid, p)
        ctx.wait(c)
        torch.cuda.synchronize()
        assert np.all(dn.cpu().numpy() == 0.0)          # identical runs
        ctx.release(c)
