"""Pins of the oracle's scalar advection physics (Sec. 3.4, Eq. 13) against
what the mathematics fixes, independent of the oracle's own formulas:

  * the numerical fluxes with the wave speeds min(v, 0), max(v, 0) reduce to
    exact upwinding (v rho_L for v > 0, v rho_R for v < 0, 0 for v = 0);
  * the time-step limit is CFL / sum_d |v_d| / dx_d;
  * translating a smooth periodic wave converges to the exact solution at
    second order with van Leer + Heun and fifth order with WENO5 + RK4
    (Sec. 4.1.2 reports the same orders);
  * the integral of the scalar is conserved to rounding on a refined mesh
    with flux fixing (Sec. 4.1.1, Eq. 18);
  * swapping the axes of the data and of the velocity swaps the result;
    mirroring x and reversing v_x mirrors it; a constant stays constant;
  * the refinement criterion on the scalar equals the Euler criterion on
    the same density at constant pressure (whose own score vanishes).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def interior(spec, u):
    S, sl = spec.side, slice(spec.ng, spec.ng + spec.N)
    a = u.reshape((u.shape[0], spec.nvar) + (S,) * spec.ndim)
    return a[(slice(None), slice(None)) + (sl,) * spec.ndim]


@pytest.mark.parametrize("flux", [0, 1])
def test_advection_flux_is_exact_upwinding(flux):
    rng = np.random.default_rng(1)
    for v in (1.3, -0.7, 0.0, 2.0 ** -30, -5.5):
        sp = synth.advection_spec(ndim=3, velocity=(v, -v, 0.5 * v))
        sp.flux = flux
        for _ in range(20):
            rL, rR = rng.normal(size=2) * 3.0
            for n in range(3):
                vn = sp.velocity[n]
                F = oracle.face_flux(sp, n, [rL], [rR])
                up = vn * (rL if vn > 0 else rR)
                assert F.shape == (1,)
                assert abs(F[0] - up) <= 4e-16 * (abs(vn) * (abs(rL) + abs(rR))), (flux, v, n, F[0], up)


def test_advection_max_speed_is_velocity_over_dx():
    sp = synth.advection_spec(ndim=3, N=8, ntrees=(2, 3, 2), velocity=(0.5, -2.0, 1.25), max_level=2)
    m = oracle.Mesh(sp, 0)
    lev, g = m.blocks()
    m = m.adapt(synth.ball_flags(sp, lev, g, (0.3, 0.4, 0.5), (0.2,)))
    lev, g = m.blocks()
    u = synth.advection_gaussian(sp, lev, g)
    L = lev.max()
    exp = sum(abs(sp.velocity[d]) / (sp.length[d] / sp.ntrees[d] / (sp.N * 2 ** L)) for d in range(3))
    assert m.max_speed(u) == pytest.approx(exp, rel=1e-15)
    assert m.dt(u) == pytest.approx(sp.cfl / exp, rel=1e-15)


def translate(n, N, limiter, scheme, T=0.25, cfl=0.5):
    sp = synth.advection_spec(ndim=2, N=N, ntrees=(n // N, n // N, 1), limiter=limiter, velocity=(1.0, 1.0))
    m = oracle.Mesh(sp, 0)
    lev, g = m.blocks()
    u = synth.advection_wave(sp, lev, g)
    dt = cfl / m.max_speed(u)
    nst = int(np.ceil(T / dt))
    for _ in range(nst):
        oracle.rk_step(m, u, scheme, dt=T / nst)
    ex = synth.advection_wave(sp, lev, g, t=T)
    return np.abs(interior(sp, u) - interior(sp, ex)).mean()


def test_advection_vanleer_heun_converges_at_second_order():
    e = [translate(n, 16, 2, "heun") for n in (32, 64, 128)]
    orders = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert np.all((orders > 1.8) & (orders < 2.3)), orders


def test_advection_weno5_rk4_converges_at_fifth_order():
    # CFL shrinks like dx^(1/4) so that RK4's dt^4 error falls like dx^5
    e = [translate(n, 16 if n >= 64 else 8, 3, "rk4", cfl=0.5 * (16.0 / n) ** 0.25) for n in (32, 64, 128)]
    orders = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert np.all(orders > 4.7), orders
    assert e[-1] < 1e-7


@pytest.mark.parametrize("ndim", [2, 3])
def test_advection_conserved_to_rounding_on_refined_mesh(ndim):
    """The flux-fixing test of Sec. 4.1.1: the smoothed sphere of Eq. 17 moves
    diagonally across refinement boundaries of a statically refined mesh;
    the conservation error of Eq. 18 stays at rounding level."""
    N = 16 if ndim == 2 else 8
    sp = synth.advection_spec(ndim=ndim, N=N, ntrees=(4,) * ndim + (1,) * (3 - ndim), limiter=2, max_level=2,
                              velocity=(1.0, 1.0, 1.0))
    m = oracle.Mesh(sp, 0)
    c = (0.62, 0.62, 0.62)
    for _ in range(2):
        lev, g = m.blocks()
        m = m.adapt(synth.ball_flags(sp, lev, g, c, (0.15, 0.08)))
    lev, g = m.blocks()
    assert lev.max() == 2 and lev.min() == 0
    u = synth.advection_sphere(sp, lev, g, R=0.2, delta=0.1)
    s0 = m.conserved(u)[0]
    for _ in range(40 if ndim == 2 else 12):
        oracle.rk_step(m, u, "heun")
    s1 = m.conserved(u)[0]
    assert abs(s1 - s0) <= 1e-14 * abs(s0), (s0, s1)
    assert interior(sp, u).max() <= 1.0 + 1e-12 and interior(sp, u).min() >= -1e-12   # TVD: no new extrema


def test_advection_axis_swap_swaps_the_result():
    out = []
    for axis in (0, 1):
        vel = (1.0, 0.0) if axis == 0 else (0.0, 1.0)
        sp = synth.advection_spec(ndim=2, N=8, ntrees=(3, 3, 1), limiter=0, velocity=vel)
        m = oracle.Mesh(sp, 0)
        lev, g = m.blocks()
        X = synth.cell_centres(sp, lev, g)
        x = X[axis]
        rho = 1.0 + 0.3 * np.sin(2 * np.pi * x) + 0.2 * np.cos(6 * np.pi * x)
        u = synth.mask_interior(sp, rho.reshape(len(rho), 1, -1).copy())
        for _ in range(5):
            oracle.rk_step(m, u, "heun")
        a = interior(sp, u)[:, 0]
        # assemble the global 24 x 24 field (block row-major, blocks of 8x8)
        G = np.zeros((24, 24))
        for b in range(m.n):
            G[8 * g[b, 1]:8 * g[b, 1] + 8, 8 * g[b, 0]:8 * g[b, 0] + 8] = a[b]
        out.append(G)
    np.testing.assert_allclose(out[0], out[1].T, rtol=0, atol=1e-15)


def test_advection_mirror_reverses_velocity():
    res = []
    for sgn in (1.0, -1.0):
        sp = synth.advection_spec(ndim=2, N=8, ntrees=(4, 2, 1), limiter=2, velocity=(0.7 * sgn, 0.3))
        m = oracle.Mesh(sp, 0)
        lev, g = m.blocks()
        X = synth.cell_centres(sp, lev, g)
        x = X[0] if sgn > 0 else 1.0 - X[0]
        rho = np.exp(-((x - 0.3) ** 2 + (X[1] - 0.6) ** 2) / 0.02)
        u = synth.mask_interior(sp, rho.reshape(len(rho), 1, -1).copy())
        for _ in range(6):
            oracle.rk_step(m, u, "heun")
        a = interior(sp, u)[:, 0]
        G = np.zeros((16, 32))
        for b in range(m.n):
            G[8 * g[b, 1]:8 * g[b, 1] + 8, 8 * g[b, 0]:8 * g[b, 0] + 8] = a[b]
        res.append(G)
    np.testing.assert_allclose(res[0], res[1][:, ::-1], rtol=0, atol=1e-15)


@pytest.mark.parametrize("limiter,flux", [(0, 0), (2, 1), (1, 0), (3, 1)])
def test_advection_constant_state_is_kept(limiter, flux):
    sp = synth.advection_spec(ndim=2, N=8, ntrees=(2, 2, 1), limiter=limiter, max_level=2, velocity=(0.4, -1.1))
    sp.flux = flux
    m = oracle.Mesh(sp, 1)
    lev, g = m.blocks()
    m = m.adapt(synth.ball_flags(sp, lev, g, (0.4, 0.4), (0.3, 0.2)))
    lev, g = m.blocks()
    u = synth.mask_interior(sp, np.full((m.n, 1, sp.ncell), 2.5))
    for scheme in ("heun", "rk4"):
        oracle.rk_step(m, u, scheme)
    assert np.all(interior(sp, u) == 2.5)


def test_advection_flags_equal_euler_flags_at_constant_pressure():
    spa = synth.advection_spec(ndim=2, N=8, ntrees=(3, 3, 1), velocity=(1.0, 1.0), max_level=1)
    spe = synth.MeshSpec(ndim=2, N=8, ng=2, ntrees=(3, 3, 1), max_level=1)
    ma, me = oracle.Mesh(spa, 1), oracle.Mesh(spe, 1)
    lev, g = ma.blocks()
    ua = synth.advection_sphere(spa, lev, g, R=0.25, delta=0.1)
    rho = ua.reshape(ma.n, -1) + 0.5
    ua = synth.mask_interior(spa, rho.reshape(ma.n, 1, -1).copy())
    ue = np.zeros((me.n, 4, spe.ncell))
    ue[:, 0] = rho
    ue[:, 3] = 1.0 / (spe.gamma - 1.0)
    ue = synth.mask_interior(spe, ue)
    ma.fill_ghosts(ua)
    me.fill_ghosts(ue)
    fa, fe = ma.lohner_flags(ua), me.lohner_flags(ue)
    np.testing.assert_array_equal(fa, fe)
    assert (fa == 1).any() and (fa == -1).any()
