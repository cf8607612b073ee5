"""Scar comparison metrics on the GPU vs the oracle (needs a GB300).

Sec. 4.1: hourly MSE and SSIM between two runs' scars and the norm of the
difference of the final scars.  The GPU evaluates them from the counts
a = |X^t|, b = |Y^t|, c = |X^t and Y^t|; the oracle from the 0-1 grids of its
own replicas (its own runs, never the GPU's).  MSE is a single rounding of an
exact integer ratio on both sides, so it is compared exactly; SSIM's oracle
sums (x - mu)^2 and (x - mu_x)(y - mu_y) over the grid, so the two differ by
rounding only: relative 1e-10 (absolute 1e-12) covers sums of 10^5-10^6 terms
with the C2 = 9e-4 floor of the numerator factor; the norm: relative 1e-14.
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


@pytest.fixture(scope="module")
def ctx():
    c2f.build()
    with c2f.Context(0) as c:
        yield c


def _oracle_metrics(w, over_x, over_y, replicas):
    L = w.landscape
    ox = oracle.Oracle(L.fuel, L.slope, L.aspect, L.unburnable, cell_size=L.cell_size,
                       weather=w.weather, **dict(w.params, **over_x))
    oy = oracle.Oracle(L.fuel, L.slope, L.aspect, L.unburnable, cell_size=L.cell_size,
                       weather=w.weather, **dict(w.params, **over_y))
    H = w.params["hours"]
    sph = 60 // w.params.get("minutes_per_step", 1)
    out = {}
    for r in replicas:
        ix, iy = ox.run_replica(r)["ign"], oy.run_replica(r)["ign"]
        mse = [oracle.scar_mse(oracle.scar_at_hour(ix, t, sph), oracle.scar_at_hour(iy, t, sph))
               for t in range(H)]
        ssim = [oracle.scar_ssim(oracle.scar_at_hour(ix, t, sph), oracle.scar_at_hour(iy, t, sph))
                for t in range(H)]
        dn = oracle.scar_dnorm(ix >= 0, iy >= 0)
        out[r] = (np.array(mse), np.array(ssim), dn)
    ox.close()
    oy.close()
    return out


def _check(got, ref, r):
    mse, ssim, dn = got
    rm, rs, rd = ref
    assert np.array_equal(mse[r], rm), (r, mse[r], rm)
    np.testing.assert_allclose(ssim[r], rs, rtol=1e-10, atol=1e-12, err_msg=str(r))
    assert dn[r] == pytest.approx(rd, rel=1e-14, abs=0.0), r


def _run_pair(ctx, w, over_x, over_y):
    L = w.landscape
    lid = ctx.load_landscape(L.fuel, L.slope, L.aspect, L.unburnable, L.cell_size)
    ctx.set_weather(lid, w.weather)
    sx = ctx.simulate(lid, _params(**dict(w.params, **over_x)))
    sy = ctx.simulate(lid, _params(**dict(w.params, **over_y)))
    return lid, sx, sy


@pytest.mark.parametrize("side,hours,mps", [(60, 4, 1), (47, 3, 10)])
def test_ellipse_variants_match_the_oracle(ctx, side, hours, mps):
    """Eq. (1) against the centre-offset ellipse ray (Sec. 3.7), every replica."""
    w = S.config2(side=side, n_replicas=10, hours=hours)
    w.params["minutes_per_step"] = mps
    lid, sx, sy = _run_pair(ctx, w, dict(ellipse_mode=0), dict(ellipse_mode=1))
    got = ctx.compare_scars(sx, sy, 10, hours)
    ref = _oracle_metrics(w, dict(ellipse_mode=0), dict(ellipse_mode=1), range(10))
    for r in range(10):
        _check(got, ref[r], r)
    assert (got[0] >= 0).all() and (got[1] <= 1.0 + 1e-15).all()
    ctx.release(lid)


def test_seeds_and_identity(ctx):
    w = S.config2(side=52, n_replicas=8, hours=3)
    lid, sx, sy = _run_pair(ctx, w, dict(seed=11), dict(seed=12))
    got = ctx.compare_scars(sx, sy, 8, 3)
    ref = _oracle_metrics(w, dict(seed=11), dict(seed=12), range(8))
    for r in range(8):
        _check(got, ref[r], r)
    mse, ssim, dn = ctx.compare_scars(sx, sx, 8, 3)
    assert (mse == 0).all() and (dn == 0).all()
    np.testing.assert_allclose(ssim, 1.0, rtol=0, atol=1e-15)
    ctx.release(lid)


def test_final_norm_without_steps_and_errors(ctx):
    w = S.config2(side=40, n_replicas=6, hours=2)
    L = w.landscape
    lid = ctx.load_landscape(L.fuel, L.slope, L.aspect, L.unburnable, L.cell_size)
    ctx.set_weather(lid, w.weather)
    plain = c2f.OUT_SCARS | c2f.OUT_COUNTERS
    sx = ctx.simulate(lid, _params(**dict(w.params, outputs=plain, ellipse_mode=0)))
    sy = ctx.simulate(lid, _params(**dict(w.params, outputs=plain, ellipse_mode=1)))
    _, _, dn = ctx.compare_scars(sx, sy, 6, 2, hourly=False)
    ref = _oracle_metrics(w, dict(ellipse_mode=0), dict(ellipse_mode=1), range(6))
    for r in range(6):
        assert dn[r] == pytest.approx(ref[r][2], rel=1e-14, abs=0.0)
    with pytest.raises(c2f.C2FError) as e:          # hourly metrics need the steps
        ctx.compare_scars(sx, sy, 6, 2)
    assert e.value.code == c2f.C2F_EINVAL
    s3 = ctx.simulate(lid, _params(**dict(w.params, n_replicas=5)))
    with pytest.raises(c2f.C2FError) as e:          # replica counts differ
        ctx.compare_scars(sx, s3, 6, 2, hourly=False)
    assert e.value.code == c2f.C2F_EINVAL
    with pytest.raises(c2f.C2FError) as e:
        ctx.compare_scars(sx, 987654, 6, 2, hourly=False)
    assert e.value.code == c2f.C2F_ENOTFOUND
    ctx.release(lid)


def test_full_size_sampled():
    """512 x 512, 24 h, 1000 replicas per variant, as the benchmark runs it;
    three replicas replayed by the oracle, and at every replica the identities
    that hold at any size (dnorm^2 = N mse at the last hour)."""
    c2f.build()
    w = S.config2(n_replicas=1000)
    L = w.landscape
    n = L.fuel.size
    with c2f.Context(0) as ctx:
        lid, sx, sy = _run_pair(ctx, w, dict(ellipse_mode=0), dict(ellipse_mode=1))
        got = ctx.compare_scars(sx, sy, 1000, 24)
        mse, ssim, dn = got
        np.testing.assert_array_equal(np.rint(dn ** 2), np.rint(mse[:, -1] * n))
        assert (ssim <= 1.0 + 1e-15).all() and (mse >= 0).all()
        ref = _oracle_metrics(w, dict(ellipse_mode=0), dict(ellipse_mode=1), (0, 499, 999))
        for r in (0, 499, 999):
            _check(got, ref[r], r)


def test_one_cell_grid_and_one_hour(ctx):
    """A 1 x 1 grid has no SSIM (1/(N-1) statistics): hourly metrics are refused,
    the final norm is 0; a 1-hour run compares its single hour."""
    fuel = np.array([[2]], dtype=np.uint8)
    lid = ctx.load_landscape(fuel, cell_size=100.0)
    ctx.set_weather(lid, S.weather_stream(1, seed=3))
    p = _params(n_replicas=3, hours=1, ignition_mode=0, ignition_cell=0)
    sx, sy = ctx.simulate(lid, p), ctx.simulate(lid, p)
    with pytest.raises(c2f.C2FError) as e:
        ctx.compare_scars(sx, sy, 3, 1)
    assert e.value.code == c2f.C2F_EINVAL
    _, _, dn = ctx.compare_scars(sx, sy, 3, 1, hourly=False)
    assert (dn == 0).all()
    ctx.release(lid)
    w = S.config2(side=20, n_replicas=4, hours=1)
    lid, sx, sy = _run_pair(ctx, w, dict(ellipse_mode=0), dict(ellipse_mode=1))
    got = ctx.compare_scars(sx, sy, 4, 1)
    ref = _oracle_metrics(w, dict(ellipse_mode=0), dict(ellipse_mode=1), range(4))
    for r in range(4):
        _check(got, ref[r], r)
    ctx.release(lid)
