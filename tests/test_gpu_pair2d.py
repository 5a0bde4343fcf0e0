"""GPU parity of the FP32 2D packed-pair stage kernel (Sec. 3.1-3.5, Eq. 5
on 2D blocks of N^2 cells, two ghost layers) against the FP64 oracle.

The kernel runs for every FP32 2D forest with two ghost layers, a MUSCL
slope limiter and the Rusanov or HLL flux unless the per-cell kernel is
chosen (launch shape >= 100).
Bars: relative L1 <= 1e-5 per variable against the oracle (the FP32 bar);
launch shapes of the pair kernel bit-identical to each other, the per-cell
FP32 kernel within FP32 rounding order (1e-6)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

amr = pytest.importorskip("paper_2605_07612_b300")

from test_gpu_parity import ball, make_pair, rel_l1, scaled_l1, SLOTS  # noqa: E402


def run(f, u, n, **kw):
    f.set_state(0, u.astype(np.float32))
    f.compute_dt(0)
    dts = []
    for _ in range(n):
        dts.append(f.get_dt())
        f.step(1, **kw)
    assert f.sync_status() == amr.AMR_OK
    return f.get_state(0), dts


@pytest.mark.parametrize("N,tile8", [(8, False), (16, False), (16, True), (32, False), (32, True)])
@pytest.mark.parametrize("gather", [False, True])
def test_pair2d_uniform_matches_oracle(N, tile8, gather):
    """Periodic Kelvin-Helmholtz on 128^2 cells, every block size and staging
    tile, halos from the ghost fill or gathered: 20 Heun steps."""
    sp = synth.MeshSpec(ndim=2, N=N, ng=2, ntrees=(128 // N, 128 // N, 1))
    om, f = make_pair(sp, 0, precision=32)
    f.set_launch_shape(1001 if tile8 else 1)
    lev, g = om.blocks()
    u = synth.kelvin_helmholtz(sp, lev, g, seed=21)
    got, dts = run(f, u, 20, gather=gather)
    ref = u.copy()
    odts = oracle.run_heun(om, ref, 20)
    np.testing.assert_allclose(dts, odts, rtol=2e-6)
    assert rel_l1(got, ref, sp).max() <= 1e-5


@pytest.mark.parametrize("N", [8, 16, 32])
def test_pair2d_amr_flux_fixing_matches_oracle(N):
    """Three levels around a ball (refinement faces: coarse-to-fine
    prolongation, restriction, flux fixing, CFL speed of the fixed cells
    taken after fixing), gathered halos and a CUDA graph: 20 Heun steps."""
    nt = 64 // N
    sp = synth.MeshSpec(ndim=2, N=N, ng=2, ntrees=(nt, nt, 1), max_level=2)
    om, f = make_pair(sp, 0, [ball((0.4, 0.55), (0.3, 0.15))] * 2, precision=32)
    lev, g = om.blocks()
    assert lev.max() == 2
    u = synth.kelvin_helmholtz(sp, lev, g, seed=22)
    got, dts = run(f, u, 20, gather=True, use_graph=True)
    ref = u.copy()
    odts = oracle.run_heun(om, ref, 20)
    np.testing.assert_allclose(dts, odts, rtol=2e-6)
    assert rel_l1(got, ref, sp).max() <= 1e-5


@pytest.mark.parametrize("limiter,flux", [(1, 0), (2, 0), (0, 1), (2, 1)])
def test_pair2d_limiters_match_oracle(limiter, flux):
    """Monotonized central and van Leer slopes, Rusanov and HLL fluxes in
    the 2D pair kernel on a Sod tube (Neumann x faces) refined around the
    diaphragm."""
    sp = synth.MeshSpec(ndim=2, N=16, ng=2, ntrees=(8, 1, 1), periodic=(0, 1, 1), max_level=1,
                        bc_type=(2, 2, 0, 0, 0, 0), length=(1.0, 1.0 / 8, 1.0), limiter=limiter, flux=flux)
    om, f = make_pair(sp, 0, [ball((0.4, 0.06), (0.1,))], precision=32)
    lev, g = om.blocks()
    u = synth.shock_tube(sp, lev, g, x0=0.4)
    got, _ = run(f, u, 20, gather=True)
    ref = u.copy()
    oracle.run_heun(om, ref, 20)
    assert rel_l1(got, ref, sp).max() <= 1e-5


@pytest.mark.parametrize("limiter", [0, 2])
def test_pair2d_rayleigh_taylor(limiter):
    """Gravity source and hydrostatic Neumann faces (Sec. 4.2 setup) in the
    2D pair kernel: L1 error <= 1e-5 of each variable's scale (momentum
    against sqrt(mass x energy)) after 20 steps."""
    sp = synth.rayleigh_taylor_spec(ndim=2, N=16, ntrees=(4, 4, 1), limiter=limiter)
    om, f = make_pair(sp, 0, precision=32)
    lev, g = om.blocks()
    u = synth.rayleigh_taylor(sp, lev, g)
    got, _ = run(f, u, 20, gather=True, use_graph=True)
    ref = u.copy()
    oracle.run_heun(om, ref, 20)
    assert scaled_l1(got, ref, sp).max() <= 1e-5


@pytest.mark.parametrize("scheme", ["ssp3", "rk4"])
def test_pair2d_rk_schemes(scheme):
    """Stages with three and more previous states take the kernel's runtime
    previous-state loop: SSP-RK3 and RK4 on a 2-level mesh."""
    sp = synth.MeshSpec(ndim=2, N=16, ng=2, ntrees=(4, 4, 1), max_level=1)
    om, f = make_pair(sp, 0, [ball((0.5, 0.5), (0.25,))], precision=32, n_states=SLOTS[scheme])
    lev, g = om.blocks()
    u = synth.kelvin_helmholtz(sp, lev, g, seed=23)
    got, _ = run(f, u, 10, gather=True, scheme=scheme)
    ref = u.copy()
    for _ in range(10):
        oracle.rk_step(om, ref, scheme)
    assert rel_l1(got, ref, sp).max() <= 1e-5


@pytest.mark.parametrize("N", [16, 32])
def test_pair2d_launch_shapes_agree(N):
    """Tiles 16 or 8, k items per CTA or a persistent grid: bit-identical;
    the per-cell kernel (the textbook flux formula, where the pair kernel
    groups the flux terms by side): within the FP32 bar against the oracle
    -- the transverse momentum of the Kelvin-Helmholtz band is a small
    perturbation whose rounding differences the instability amplifies."""
    sp = synth.MeshSpec(ndim=2, N=N, ng=2, ntrees=(256 // N, 256 // N, 1), max_level=1)
    f = amr.Forest(sp, 0, max_blocks=4 * (256 // N) ** 2, precision=32)
    lev, g = f.blocks()
    f.regrid(synth.ball_flags(sp, lev, g, (0.5, 0.5), (0.2,)))
    lev, g = f.blocks()
    u = synth.kelvin_helmholtz(sp, lev, g, seed=24).astype(np.float32)
    results = {}
    for choice in (1, 2, 4, 0, 1001, 1002, 1000, 101, 100):
        f.set_launch_shape(choice)
        f.set_state(0, u)
        f.compute_dt(0)
        f.step(4, use_graph=True, gather=True)
        assert f.sync_status() == amr.AMR_OK
        results[choice] = f.get_state(0)
    for c in (2, 4, 0, 1001, 1002, 1000):
        np.testing.assert_array_equal(results[c], results[1])
    for c in (101, 100):
        assert rel_l1(results[c], results[1].astype(np.float64), sp).max() <= 1e-5


def test_pair2d_nonphysical_state_is_reported():
    sp = synth.MeshSpec(ndim=2, N=16, ng=2, ntrees=(2, 2, 1))
    f = amr.Forest(sp, 0, precision=32)
    lev, g = f.blocks()
    u = synth.kelvin_helmholtz(sp, lev, g).astype(np.float32)
    u.reshape(f.n, sp.nvar, sp.side, sp.side)[1, 3, 7, 9] = -1.0     # negative energy -> pressure
    f.set_state(0, u)
    f.set_dt(1e-4)
    f.step(1, gather=True)
    assert f.sync_status() == amr.AMR_ENONPHYS
    assert f.sync_status() == amr.AMR_OK


@pytest.mark.parametrize("flux", [0, 1])
def test_pair2d_kernels_agree_with_per_cell_kernel(flux):
    """The pair kernel (either flux) and the per-cell kernel on a 2-level
    mesh: each within the FP32 bar of the oracle, and within FP32 rounding
    order of each other measured against each variable's scale (the
    y-momentum of this flow is only the seeded perturbation, so its own L1
    norm is not a meaningful scale)."""
    sp = synth.MeshSpec(ndim=2, N=16, ng=2, ntrees=(8, 8, 1), max_level=1, limiter=2, flux=flux)
    om, f = make_pair(sp, 0, [ball((0.5, 0.5), (0.25,))], precision=32)
    lev, g = f.blocks()
    u = synth.kelvin_helmholtz(sp, lev, g, seed=25)
    res = {}
    for choice in (1, 101):
        f.set_launch_shape(choice)
        f.set_state(0, u.astype(np.float32))
        f.compute_dt(0)
        f.step(6, use_graph=True, gather=True)
        assert f.sync_status() == amr.AMR_OK
        res[choice] = f.get_state(0).astype(np.float64)
    ref = u.copy()
    oracle.run_heun(om, ref, 6)
    for c in (1, 101):
        assert rel_l1(res[c], ref, sp).max() <= 1e-5
    assert scaled_l1(res[101], res[1], sp).max() <= 1e-6
