"""Pins of the oracle's further face reconstructions of Sec. 3.2 (Koren,
WENO3, first-order upwind) against what the mathematics fixes:

  * Koren's limiter reproduces the third-order (kappa = 1/3) face value
    (-w_{i-1} + 5 w_i + 2 w_{i+1}) / 6 -- exact for cell averages of a
    quadratic -- wherever the ratio of differences lies in (1/4, 5/2), and
    keeps every face value between the cell and its neighbour (TVD);
  * WENO3 is exact on linear data and reduces to the same third-order value
    when both stencils are equally smooth;
  * first-order upwind uses the cell values;
  * translating a smooth wave converges at order 1 (upwind) and about 2
    (Koren, WENO3; limited at the extrema), and Koren and upwind create no
    new extrema.
"""
import numpy as np
import pytest

import oracle
import synth

from test_oracle_advection import interior, translate

KOREN, WENO3, UPWIND = 4, 5, 6


def test_koren_is_third_order_on_quadratics():
    rng = np.random.default_rng(11)
    n = 0
    while n < 200:
        c0, c1, c2 = rng.normal(size=3)
        # cell averages over [i - 1/2, i + 1/2] of c0 + c1 x + c2 x^2
        avg = lambda i: c0 + c1 * i + c2 * (i * i + 1.0 / 12.0)
        f = lambda x: c0 + c1 * x + c2 * x * x
        wm, w0, wp = avg(-1), avg(0), avg(1)
        a, b = w0 - wm, wp - w0
        if not (0.25 < b / a < 2.5 and 0.25 < a / b < 2.5):
            continue
        lo, hi = oracle.cell_faces(KOREN, wm, w0, wp)
        assert hi == pytest.approx(f(0.5), rel=1e-13, abs=1e-13)
        assert lo == pytest.approx(f(-0.5), rel=1e-13, abs=1e-13)
        n += 1


def test_koren_face_values_stay_between_neighbours():
    rng = np.random.default_rng(12)
    for _ in range(2000):
        wm, w0, wp = rng.normal(size=3) * rng.choice([1e-3, 1.0, 1e3])
        lo, hi = oracle.cell_faces(KOREN, wm, w0, wp)
        assert min(w0, wp) - 1e-12 * abs(w0) <= hi <= max(w0, wp) + 1e-12 * abs(w0)
        assert min(w0, wm) - 1e-12 * abs(w0) <= lo <= max(w0, wm) + 1e-12 * abs(w0)
        if (w0 - wm) * (wp - w0) <= 0:          # a local extremum: first order
            assert lo == w0 and hi == w0


def test_weno3_exact_on_linear_data_and_third_order_when_smooth():
    rng = np.random.default_rng(13)
    for _ in range(100):
        c0, c1 = rng.normal(size=2)
        lo, hi = oracle.cell_faces(WENO3, c0 - c1, c0, c0 + c1)
        assert hi == pytest.approx(c0 + 0.5 * c1, rel=1e-13, abs=1e-13)
        assert lo == pytest.approx(c0 - 0.5 * c1, rel=1e-13, abs=1e-13)
    # equal smoothness of both stencils (|a| = |b|): the linear weights, i.e.
    # the kappa = 1/3 value
    for wm, w0, wp in ((0.0, 1.0, 0.0), (2.0, 1.0, 2.0), (0.5, 1.5, 2.5)):
        lo, hi = oracle.cell_faces(WENO3, wm, w0, wp)
        assert hi == pytest.approx((-wm + 5 * w0 + 2 * wp) / 6.0, rel=1e-12)
        assert lo == pytest.approx((-wp + 5 * w0 + 2 * wm) / 6.0, rel=1e-12)


def test_upwind_uses_cell_values():
    for wm, w0, wp in ((0.0, 1.0, 3.0), (-1.0, 2.0, -5.0)):
        assert oracle.cell_faces(UPWIND, wm, w0, wp) == (w0, w0)


@pytest.mark.parametrize("lim,lo_order,hi_order", [(UPWIND, 0.8, 1.1), (KOREN, 1.95, 2.5), (WENO3, 1.9, 2.6)])
def test_translation_convergence_orders(lim, lo_order, hi_order):
    e = [translate(n, 16, lim, "heun") for n in (32, 64, 128)]
    orders = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert np.all((orders > lo_order) & (orders < hi_order)), orders


@pytest.mark.parametrize("lim", [KOREN, UPWIND])
def test_no_new_extrema(lim):
    sp = synth.advection_spec(ndim=2, N=16, ntrees=(4, 4, 1), limiter=lim, velocity=(1.0, 0.7))
    m = oracle.Mesh(sp, 0)
    lev, g = m.blocks()
    u = synth.advection_sphere(sp, lev, g, R=0.2, delta=0.02)
    for _ in range(30):
        oracle.rk_step(m, u, "heun")
    a = interior(sp, u)
    assert a.max() <= 1.0 + 1e-13 and a.min() >= -1e-13
