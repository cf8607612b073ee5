"""Oracle pins: fire-scar comparison metrics (Sec. 4.1).

MSE, SSIM (Wang et al.'s single-window form, C1 = 0.01^2, C2 = 0.03^2, 1/(N-1)
statistics; the printed second denominator factor read as sigma_X^2 +
sigma_Y^2 + C2) and the Frobenius norm of X - Y.  Pinned by closed forms in
the counts a = |X|, b = |Y|, c = |X and Y| of two 0-1 scars, by special cases
(identical, complementary, empty and full scars) and by invariants
(symmetry, SSIM <= 1).
"""
import math

import numpy as np
import pytest

import oracle


def _counts(x, y):
    x = np.asarray(x, dtype=bool)
    y = np.asarray(y, dtype=bool)
    return int(x.sum()), int(y.sum()), int((x & y).sum()), x.size


def _ssim_counts(a, b, c, n):
    # the same statistics derived by hand for 0-1 data
    mx, my = a / n, b / n
    vx = a * (n - a) / (n * (n - 1))
    vy = b * (n - b) / (n * (n - 1))
    cxy = (c * n - a * b) / (n * (n - 1))
    c1, c2 = 0.01 ** 2, 0.03 ** 2
    return (2 * mx * my + c1) * (2 * cxy + c2) / ((mx * mx + my * my + c1) * (vx + vy + c2))


@pytest.mark.parametrize("seed", range(6))
def test_closed_forms_in_the_counts(seed):
    rng = np.random.default_rng(seed)
    shape = tuple(rng.integers(3, 40, 2))
    x = rng.random(shape) < rng.uniform(0.05, 0.9)
    y = x.copy()
    flip = rng.random(shape) < rng.uniform(0.0, 0.4)
    y[flip] = ~y[flip]
    a, b, c, n = _counts(x, y)
    assert oracle.scar_mse(x, y) == pytest.approx((a + b - 2 * c) / n, rel=1e-14, abs=1e-15)
    assert oracle.scar_dnorm(x, y) == pytest.approx(math.sqrt(a + b - 2 * c), rel=1e-14, abs=1e-15)
    assert oracle.scar_ssim(x, y) == pytest.approx(_ssim_counts(a, b, c, n), rel=1e-12)


def test_identical_and_complementary_scars():
    rng = np.random.default_rng(7)
    x = rng.random((25, 31)) < 0.3
    assert oracle.scar_mse(x, x) == 0.0 and oracle.scar_dnorm(x, x) == 0.0
    assert oracle.scar_ssim(x, x) == pytest.approx(1.0, abs=1e-15)
    y = ~x
    assert oracle.scar_mse(x, y) == 1.0
    assert oracle.scar_dnorm(x, y) == pytest.approx(math.sqrt(x.size), rel=1e-15)
    # perfectly anti-correlated: sigma_xy = -sigma_x sigma_y
    a, b, c, n = _counts(x, y)
    assert oracle.scar_ssim(x, y) == pytest.approx(_ssim_counts(a, b, c, n), rel=1e-12)
    assert oracle.scar_ssim(x, y) < 0.0


def test_empty_and_full_scars():
    z = np.zeros((10, 12))
    o = np.ones((10, 12))
    assert oracle.scar_ssim(z, z) == pytest.approx(1.0, abs=1e-15)   # C1 C2 / (C1 C2)
    c1 = 0.01 ** 2
    assert oracle.scar_ssim(o, z) == pytest.approx(c1 / (1.0 + c1), rel=1e-12)
    assert oracle.scar_mse(o, z) == 1.0


def test_symmetry_and_bound():
    rng = np.random.default_rng(9)
    for _ in range(20):
        x = rng.random((17, 19)) < rng.uniform(0, 1)
        y = rng.random((17, 19)) < rng.uniform(0, 1)
        assert oracle.scar_ssim(x, y) == pytest.approx(oracle.scar_ssim(y, x), rel=1e-14)
        assert oracle.scar_ssim(x, y) <= 1.0 + 1e-15


def test_printed_denominator_would_not_give_one():
    """The reading: with the printed factor mu_x^2 + mu_y^2 + C2 in place of
    sigma_x^2 + sigma_y^2 + C2, identical scars would not score 1."""
    rng = np.random.default_rng(3)
    x = (rng.random((20, 20)) < 0.4).astype(np.float64)
    mx = x.mean()
    vx = x.var(ddof=1)
    c1, c2 = 0.01 ** 2, 0.03 ** 2
    printed = (2 * mx * mx + c1) * (2 * vx + c2) / ((2 * mx * mx + c1) * (2 * mx * mx + c2))
    assert abs(printed - 1.0) > 0.1
    assert oracle.scar_ssim(x, x) == pytest.approx(1.0, abs=1e-15)


def test_scar_at_hour_boundaries():
    steps = np.array([-1, 0, 1, 60, 61, 120, 121, 179, 180])
    assert list(oracle.scar_at_hour(steps, 0, 60)) == [0, 1, 1, 1, 0, 0, 0, 0, 0]
    assert list(oracle.scar_at_hour(steps, 1, 60)) == [0, 1, 1, 1, 1, 1, 0, 0, 0]
    assert list(oracle.scar_at_hour(steps, 2, 60)) == [0, 1, 1, 1, 1, 1, 1, 1, 1]
    assert list(oracle.scar_at_hour(steps, 0, 6)) == [0, 1, 1, 0, 0, 0, 0, 0, 0]
