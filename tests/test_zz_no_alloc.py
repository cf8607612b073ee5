"""c2f_frontier_static: the allocation-free frontier entry point (needs a GPU).

Callers that cannot allocate device memory (under a host application that has
handed all device memory to its own allocator, in a plugin that may not
allocate after start-up) get the frontier step from this entry point, which
takes its scratch from a fixed array inside the library.  Its results must
equal the regular c2f_simulate path exactly, call after call: with the
default options, with a receive threshold, a delta burn-out and a
burning-hours limit, and on a fire whose burning list outgrows the first
attempt's capacity so that the replicas are re-run with the whole array.
This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

import c2f_synth as S
import paper_1905_09317_gb300 as c2f

pytestmark = pytest.mark.gpu


def _pack_rows(bits2d):
    """(rows, cols) 0/1 -> rows * ceil(cols/32) uint32 words, bit c%32 of word c//32."""
    rows, cols = bits2d.shape
    wpr = (cols + 31) // 32
    padded = np.zeros((rows, wpr * 32), dtype=np.uint64)
    padded[:, :cols] = bits2d
    w = padded.reshape(rows, wpr, 32) << np.arange(32, dtype=np.uint64)
    return w.sum(axis=2).astype(np.uint32)


def _unpack_rows(words, cols):
    rows, wpr = words.shape
    bits = (words[:, :, None].astype(np.uint64) >> np.arange(32, dtype=np.uint64)) & 1
    return bits.reshape(rows, wpr * 32)[:, :cols].astype(np.uint8)


def _static_twice(p, rows, cols, cell_size, t_burn, t_base, t_hros, t_ign, ref_scars, ref_work, ref_nign):
    """Two c2f_frontier_static calls in a row, each equal to c2f_simulate's results."""
    import torch
    dev = t_burn.device
    R = p.n_replicas
    wpr = (cols + 31) // 32
    stream = torch.cuda.current_stream(dev)
    lib = c2f.load_library()
    for call in range(2):
        t_scars = torch.full((R, rows, wpr), -1, dtype=torch.int32, device=dev)
        t_work = torch.full((R,), -1, dtype=torch.int64, device=dev)
        t_nign = torch.full((R,), -1, dtype=torch.int32, device=dev)
        io = c2f.FrontierIO(rows, cols, float(cell_size), t_burn.data_ptr(), t_base.data_ptr(),
                            t_hros.data_ptr(), t_ign.data_ptr(), t_scars.data_ptr(),
                            t_work.data_ptr(), t_nign.data_ptr())
        rc = lib.c2f_frontier_static(C.byref(io), C.byref(p), C.c_void_p(stream.cuda_stream))
        assert rc == c2f.C2F_OK, (call, rc)
        torch.cuda.synchronize(dev)
        work = t_work.cpu().numpy()
        nign = t_nign.cpu().numpy()
        words = t_scars.cpu().numpy().view(np.uint32)
        scars = np.stack([_unpack_rows(words[r], cols).ravel() for r in range(R)])
        assert np.array_equal(work, ref_work), call
        assert np.array_equal(nign, ref_nign), call
        assert np.array_equal(scars, ref_scars), call


@pytest.mark.parametrize("variant", [
    dict(),                                               # the workload's own options
    dict(ros_threshold=2.5),                              # receive test HROS * f > 2.5
    dict(burnout_delta=1.5),                              # A5 (i): Burned when HROS * f < 1.5
    dict(burn_hours_min=2, burn_hours_max=5),             # A5 general (1): 2..5 burning hours a day
], ids=["default", "threshold", "delta", "burn_hours"])
def test_static_frontier_matches_simulate_twice(variant):
    torch = pytest.importorskip("torch")
    c2f.build()
    w = S.config2(side=101, n_replicas=40, hours=6)
    L = w.landscape
    rows, cols = L.fuel.shape
    n = rows * cols
    keys = {f[0] for f in c2f.SimParams._fields_}
    p = c2f.default_params(**{k: v for k, v in dict(w.params, **variant).items() if k in keys})
    R, H = p.n_replicas, p.hours
    with c2f.Context(0) as ctx:
        lid = ctx.load_landscape(L.fuel, L.slope, L.aspect, cell_size=L.cell_size)
        ctx.set_weather(lid, w.weather)
        sid = ctx.simulate(lid, p)
        ref_scars, _ = ctx.get_scars(sid, R, n)
        ref_work, ref_nign, ign_cell = ctx.get_counters(sid, R)
        base = np.empty((H, n, 8), dtype=np.int64)
        hros = np.empty((H, n), dtype=np.float64)
        for h in range(H):
            _, hros[h], base[h] = ctx.get_ros(lid, p, h, n)
    dev = torch.device("cuda", 0)
    t_burn = torch.from_numpy(_pack_rows(L.fuel != 0).view(np.int32)).to(dev)
    _static_twice(p, rows, cols, L.cell_size, t_burn, torch.from_numpy(base).to(dev),
                  torch.from_numpy(hros).to(dev), torch.from_numpy(ign_cell).to(dev),
                  ref_scars, ref_work, ref_nign)


def _max_burning(ign, shape, periods):
    """Largest number of cells burning at the start of a fire period, from one
    replica's ignition steps: a cell ignited at t burns from period t + 1
    through the period in which its last neighbour ignites (A5 (ii))."""
    rows, cols = shape
    t = ign.reshape(shape).astype(np.int64)
    tt = np.where(t < 0, 1 << 40, t)
    pad = np.pad(tt, 1, constant_values=-1)
    last = np.full(shape, -1, dtype=np.int64)
    for dr in (-1, 0, 1):
        for dc in (-1, 0, 1):
            if dr or dc:
                last = np.maximum(last, pad[1 + dr:1 + dr + rows, 1 + dc:1 + dc + cols])
    lit = t >= 0
    start, end = t[lit] + 1, np.minimum(last, periods)[lit] + 1
    d = np.zeros(periods + 3, dtype=np.int64)
    np.add.at(d, start, 1)
    np.add.at(d, np.maximum(end, start), -1)
    return int(np.cumsum(d).max())


def test_static_frontier_rerun_after_list_overflow_matches_simulate():
    """A fire with more than 4096 cells burning at once (a 1301 x 1301 open
    grid of 1 m cells at 1.5 m/min for 10 h: the front is a ring of about 4,800
    burning cells) overflows the first attempt's burning lists; those replicas
    are re-run with one slot holding the whole array, and the results still
    equal c2f_simulate's, on two calls in a row."""
    torch = pytest.importorskip("torch")
    c2f.build()
    side, hours, R, ros = 1301, 10, 3, 1.5
    n = side * side
    fuel = np.ones((side, side), dtype=np.uint8)
    p = c2f.default_params(seed=77, n_replicas=R, hours=hours, ignition_mode=0,
                           ignition_cell=(side // 2) * side + side // 2, ros_sigma=0.1, const_ros=ros,
                           outputs=c2f.OUT_SCARS | c2f.OUT_COUNTERS | c2f.OUT_IGN_STEPS)
    with c2f.Context(0) as ctx:
        lid = ctx.load_landscape(fuel, cell_size=1.0)
        ctx.set_weather(lid, S.constant_weather(hours, ws=0.0))
        sid = ctx.simulate(lid, p)
        ref_scars, ign = ctx.get_scars(sid, R, n, ign_steps=True)
        ref_work, ref_nign, ign_cell = ctx.get_counters(sid, R)
        _, hros0, base0 = ctx.get_ros(lid, p, 0, n)
    assert max(_max_burning(ign[r], (side, side), hours * 60) for r in range(R)) > 4096
    # the table is the same every hour: B_k = llrint(1.5 * 2^32) on every axis, HROS 1.5
    assert np.all(base0 == int(round(ros * 2 ** 32))) and np.all(hros0 == ros)
    dev = torch.device("cuda", 0)
    t_base = torch.full((hours, n, 8), int(round(ros * 2 ** 32)), dtype=torch.int64, device=dev)
    t_hros = torch.full((hours, n), ros, dtype=torch.float64, device=dev)
    t_burn = torch.from_numpy(_pack_rows(fuel != 0).view(np.int32)).to(dev)
    _static_twice(p, side, side, 1.0, t_burn, t_base, t_hros, torch.from_numpy(ign_cell).to(dev),
                  ref_scars, ref_work, ref_nign)


def test_static_frontier_rejects_bad_ignition_cells():
    torch = pytest.importorskip("torch")
    c2f.build()
    dev = torch.device("cuda", 0)
    rows, cols, H = 20, 40, 1
    fuel = np.ones((rows, cols), dtype=np.uint8)
    fuel[0, 5] = 0
    t_burn = torch.from_numpy(_pack_rows(fuel != 0).view(np.int32)).to(dev)
    t_base = torch.full((H, rows * cols, 8), 10 << 32, dtype=torch.int64, device=dev)
    t_hros = torch.full((H, rows * cols), 10.0, dtype=torch.float64, device=dev)
    t_scars = torch.zeros((2, rows, 2), dtype=torch.int32, device=dev)
    t_work = torch.zeros(2, dtype=torch.int64, device=dev)
    t_nign = torch.zeros(2, dtype=torch.int32, device=dev)
    lib = c2f.load_library()
    p = c2f.default_params(n_replicas=2, hours=H)
    for bad in (-1, rows * cols, 5):                      # below, past the end, non-fuel
        t_ign = torch.tensor([3, bad], dtype=torch.int32, device=dev)
        io = c2f.FrontierIO(rows, cols, 100.0, t_burn.data_ptr(), t_base.data_ptr(), t_hros.data_ptr(),
                            t_ign.data_ptr(), t_scars.data_ptr(), t_work.data_ptr(), t_nign.data_ptr())
        rc = lib.c2f_frontier_static(C.byref(io), C.byref(p),
                                     C.c_void_p(torch.cuda.current_stream(dev).cuda_stream))
        assert rc == c2f.C2F_EINVAL, bad
    p_bad = c2f.default_params(n_replicas=2, hours=H, burn_hours_min=5, burn_hours_max=3)
    io = c2f.FrontierIO(rows, cols, 100.0, t_burn.data_ptr(), t_base.data_ptr(), t_hros.data_ptr(),
                        t_scars.data_ptr(), t_scars.data_ptr(), t_work.data_ptr(), t_nign.data_ptr())
    assert lib.c2f_frontier_static(C.byref(io), C.byref(p_bad), None) == c2f.C2F_EINVAL


def test_static_frontier_rejects_oversized_landscapes():
    c2f.build()
    lib = c2f.load_library()
    p = c2f.default_params(n_replicas=1, hours=1)
    fake = 256   # any non-null device-looking value: rejected before any device work
    io = c2f.FrontierIO(65535, 65535, 100.0, fake, fake, fake, fake, fake, fake, fake)
    assert lib.c2f_frontier_static(C.byref(io), C.byref(p), None) == c2f.C2F_EINVAL
    io = c2f.FrontierIO(10, 10, 100.0, None, fake, fake, fake, fake, fake, fake)
    assert lib.c2f_frontier_static(C.byref(io), C.byref(p), None) == c2f.C2F_EINVAL
    p2 = c2f.default_params(n_replicas=70000, hours=1)
    io = c2f.FrontierIO(10, 10, 100.0, fake, fake, fake, fake, fake, fake, fake)
    assert lib.c2f_frontier_static(C.byref(io), C.byref(p2), None) == c2f.C2F_EINVAL
