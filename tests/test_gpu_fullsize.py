"""Full-size workloads, sampled replicas vs the oracle (needs a GB300).

Each workload runs at its full size in the launch configuration the
benchmark times; a sample of replicas is replayed one by one by the oracle
(replicas are independent, Sec. 3.1, and every random draw is keyed by
(seed, replica, cell, hour), so any replica can be replayed alone).  Checked
bit for bit: the replica's final burn grid, its ignition cell, its ignited
count and its work count W = sum over fire periods of the burning cells
(which depends on every ignition time).
"""
import numpy as np
import pytest

import c2f_synth as S
import oracle
import paper_1905_09317_gb300 as c2f

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

_KEYS = {f[0] for f in c2f.SimParams._fields_}


def _params(w, **over):
    d = {k: v for k, v in w.params.items() if k in _KEYS}
    d.update(over)
    return c2f.default_params(**d)


def _check_replica(ctx, sid, w, r, work, nign, ign_cell):
    L = w.landscape
    o = oracle.Oracle(L.fuel, L.slope, L.aspect, L.unburnable, cell_size=L.cell_size,
                      weather=w.weather, **w.params)
    ref = o.run_replica(r)
    scar, _ = ctx.get_replica_scar(sid, r, L.fuel.size)
    assert ign_cell[r] == ref["ignition_cell"], r
    assert work[r] == ref["work"], (r, work[r], ref["work"])
    assert nign[r] == ref["n_ignited"], r
    assert np.array_equal(scar, ref["scar"].ravel()), r
    o.close()


def test_batch_of_64_landscapes_sampled():
    """64 landscapes, 41,489 replicas, 48 h, one batched call (autotuned
    launch shape, table builds overlapping the frontier groups)."""
    c2f.build()
    specs = S.config3_specs()
    ws = [S.config3_workload(sp) for sp in specs]
    with c2f.Context(0) as ctx:
        lids = []
        for w in ws:
            L = w.landscape
            lid = ctx.load_landscape(L.fuel, L.slope, L.aspect, cell_size=L.cell_size)
            ctx.set_weather(lid, w.weather)
            lids.append(lid)
        ps = [_params(w) for w in ws]
        ctx.autotune(lids, ps, sample_replicas=4096)
        sids = ctx.simulate_batch(lids, ps)
        order = np.argsort([sp["side"] for sp in specs])
        picks = list(order[-3:]) + list(order[:2]) + [int(order[len(order) // 2])]
        for i in picks:
            w, sid, p = ws[i], sids[i], ps[i]
            work, nign, ign_cell = ctx.get_counters(sid, p.n_replicas)
            for r in sorted({0, p.n_replicas // 2, p.n_replicas - 1}):
                _check_replica(ctx, sid, w, r, work, nign, ign_cell)
            counts = ctx.burn_prob(sid, w.landscape.fuel.size)
            assert counts.max() <= p.n_replicas and counts.sum() == nign.sum()


def test_large_landscape_4096_sampled():
    """4096 x 4096 cells, 72 h with a 90-degree wind shift, 256 replicas."""
    c2f.build()
    w = S.config4()
    L = w.landscape
    with c2f.Context(0) as ctx:
        lid = ctx.load_landscape(L.fuel, L.slope, L.aspect, cell_size=L.cell_size)
        ctx.set_weather(lid, w.weather)
        p = _params(w)
        sid = ctx.simulate(lid, p)
        work, nign, ign_cell = ctx.get_counters(sid, 256)
        for r in (0, 97, 255):
            _check_replica(ctx, sid, w, r, work, nign, ign_cell)
        counts = ctx.burn_prob(sid, L.fuel.size)
        assert counts.sum() == nign.sum()


def test_served_request_stream_sampled():
    """The first requests of the Poisson stream (pool landscapes of 128..2048
    cells a side, 32..2048 replicas, 12..72 h), served with continuous
    batching; one replica of every third request replayed by the oracle."""
    c2f.build()
    sides, reqs = S.serving_requests()
    reqs = reqs[:24]
    lands, weathers, lids = {}, {}, {}
    with c2f.Context(0) as ctx:
        ctx.set_serving(max_inflight=3)
        sids = []
        for q in reqs:
            k = q["pool_index"]
            if k not in lids:
                lands[k] = S.heterogeneous_landscape(sides[k], seed=500 + k)
                weathers[k] = S.weather_stream(72, seed=600 + k)
                L = lands[k]
                lids[k] = ctx.load_landscape(L.fuel, L.slope, L.aspect, cell_size=L.cell_size)
                ctx.set_weather(lids[k], weathers[k])
            p = c2f.default_params(seed=q["seed"], n_replicas=q["n_replicas"], hours=q["hours"],
                                   ignition_mode=1, ros_sigma=0.1)
            sids.append(ctx.submit(lids[k], p))
        for j in range(0, len(reqs), 3):
            q = reqs[j]
            ctx.wait(sids[j])
            k = q["pool_index"]
            w = S.Workload(lands[k], weathers[k],
                           dict(seed=q["seed"], n_replicas=q["n_replicas"], hours=q["hours"],
                                minutes_per_step=1, ignition_mode=1, ignition_cell=0, ros_sigma=0.1))
            work, nign, ign_cell = ctx.get_counters(sids[j], q["n_replicas"])
            _check_replica(ctx, sids[j], w, q["n_replicas"] - 1 - j % q["n_replicas"], work, nign, ign_cell)
        for s in sids:
            ctx.wait(s)


def test_headline_pipelined_steps_sampled():
    """The benchmark's headline configuration exactly: the 512x512 landscape,
    1000 replicas, 24 h; the frontier's shared memory sized for 8 warps per SM
    (one more than a step's replicas need), three steps in flight through
    submit / wait, each step's table rebuilt (K1) while the previous step's
    frontier runs, burn counts into device memory.  Every step's counts equal
    the sum of its scars, the steps agree with each other (same seed, same
    replicas), and replicas 0, 333, 666, 999 of each are replayed by the oracle."""
    torch = pytest.importorskip("torch")
    c2f.build()
    w = S.config2()
    L = w.landscape
    n = L.fuel.size
    p = _params(w)
    R = p.n_replicas
    with c2f.Context(0) as ctx:
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        ctx.set_frontier_config(32, -(-R // sms) + 1)
        stream = torch.cuda.Stream()
        ctx.set_stream(stream.cuda_stream)
        lid = ctx.load_landscape(L.fuel, L.slope, L.aspect, cell_size=L.cell_size)
        ctx.set_weather(lid, w.weather)
        ctx.set_serving(max_inflight=3, max_epoch_replicas=R, hbm_reserve_bytes=0)
        counts_dev = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in range(5)]
        inflight, done = [], []
        for i in range(5):
            ctx.build_ros(lid, p, force=1)
            inflight.append((i, ctx.submit(lid, p)))
            if len(inflight) >= 3:
                j, sid = inflight.pop(0)
                ctx.wait(sid)
                ctx.burn_prob_device(sid, counts_dev[j].data_ptr())
                done.append((j, sid))
        while inflight:
            j, sid = inflight.pop(0)
            ctx.wait(sid)
            ctx.burn_prob_device(sid, counts_dev[j].data_ptr())
            done.append((j, sid))
        torch.cuda.synchronize()
        first = None
        for j, sid in done:
            work, nign, ign_cell = ctx.get_counters(sid, R)
            scars, _ = ctx.get_scars(sid, R, n)
            counts = counts_dev[j].cpu().numpy().view(np.uint32)
            assert np.array_equal(counts, scars.sum(0, dtype=np.uint32)), j
            if first is None:
                first = (work, nign, ign_cell, counts)
                for r in (0, 333, 666, 999):
                    _check_replica(ctx, sid, w, r, work, nign, ign_cell)
            else:
                for a, b in zip(first, (work, nign, ign_cell, counts)):
                    assert np.array_equal(a, b), j
