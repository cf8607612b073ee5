"""c2f_frontier_static: the allocation-free frontier entry point (needs a GPU).

Callers that cannot allocate device memory (inside someone else's CUDA-graph
capture, under a host allocator that owns all device memory, in a plugin that
may not allocate after start-up) get the frontier step from this entry point,
which takes its scratch from a fixed array inside the library.  Its results
must equal the regular c2f_simulate path exactly, call after call.  This file
is collected last on purpose.
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


def test_static_frontier_matches_simulate_twice():
    torch = pytest.importorskip("torch")
    c2f.build()
    w = S.config2(side=101, n_replicas=40, hours=6)
    L = w.landscape
    rows, cols = L.fuel.shape
    n = rows * cols
    keys = {f[0] for f in c2f.SimParams._fields_}
    p = c2f.default_params(**{k: v for k, v in w.params.items() if k in keys})
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
    burn = _pack_rows(L.fuel != 0)
    t_burn = torch.from_numpy(burn.view(np.int32)).to(dev)
    t_base = torch.from_numpy(base).to(dev)
    t_hros = torch.from_numpy(hros).to(dev)
    t_ign = torch.from_numpy(ign_cell).to(dev)
    wpr = (cols + 31) // 32
    stream = torch.cuda.current_stream(dev)
    lib = c2f.load_library()
    for call in range(2):
        t_scars = torch.full((R, rows, wpr), -1, dtype=torch.int32, device=dev)
        t_work = torch.full((R,), -1, dtype=torch.int64, device=dev)
        t_nign = torch.full((R,), -1, dtype=torch.int32, device=dev)
        io = c2f.FrontierIO(rows, cols, float(L.cell_size), t_burn.data_ptr(), t_base.data_ptr(),
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
