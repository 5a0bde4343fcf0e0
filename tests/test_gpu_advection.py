"""GPU parity of the scalar advection path (Sec. 3.4, Eq. 13; the test cases
of Sec. 4.1) through the C ABI against the FP64 oracle.

Bars: FP64 relative L1 <= 1e-12 and dt within 1e-13; FP32 relative L1 <=
1e-5 after 20 steps; the conservation error of Eq. 18 at rounding level on
a refined mesh; refinement flags on the scalar bit-exact in FP64."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

amr = pytest.importorskip("paper_2605_07612_b300")

from test_gpu_parity import make_pair, rel_l1  # noqa: E402


def refined(ndim, N, limiter=2, flux=0, velocity=(1.0, 1.0, 1.0), nt=4):
    sp = synth.advection_spec(ndim=ndim, N=N, ntrees=(nt,) * ndim + (1,) * (3 - ndim), limiter=limiter,
                              velocity=velocity, max_level=2)
    sp.flux = flux
    c = (0.62, 0.58, 0.6)
    fl = lambda s, lev, g: synth.ball_flags(s, lev, g, c, (0.2, 0.1))
    return sp, [fl, fl]


def run(f, u, n, scheme="heun", **kw):
    f.set_state(0, u)
    f.compute_dt(0)
    dts = []
    for _ in range(n):
        dts.append(f.get_dt())
        f.step(1, scheme=scheme, **kw)
    assert f.sync_status() == amr.AMR_OK
    return f.get_state(0), dts


@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("limiter,flux", [(2, 0), (0, 1), (1, 0), (4, 0), (5, 1), (6, 0)])
@pytest.mark.parametrize("gather", [False, True])
def test_advection_fp64_amr_matches_oracle(ndim, limiter, flux, gather):
    sp, rounds = refined(ndim, 16 if ndim == 2 else 8, limiter, flux, velocity=(1.0, -0.6, 0.8))
    om, f = make_pair(sp, 0, rounds)
    lev, g = om.blocks()
    assert lev.max() == 2
    u = synth.advection_sphere(sp, lev, g, R=0.2, delta=0.1)
    n = 12 if ndim == 2 else 6
    got, dts = run(f, u.copy(), n, gather=gather, use_graph=gather)
    ref = u.copy()
    odts = oracle.run_heun(om, ref, n)
    np.testing.assert_allclose(dts, odts, rtol=1e-13)
    assert rel_l1(got, ref, sp).max() <= 1e-12


@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("flux", [0, 1])
def test_advection_weno5_rk4_fp64_matches_oracle(ndim, flux):
    sp, rounds = refined(ndim, 16 if ndim == 2 else 8, 3, flux, velocity=(0.5, 1.0, -1.0))
    om, f = make_pair(sp, 0, rounds, n_states=4)
    lev, g = om.blocks()
    u = synth.advection_gaussian(sp, lev, g, R=0.15)
    n = 6 if ndim == 2 else 3
    got, dts = run(f, u.copy(), n, scheme="rk4")
    ref = u.copy()
    odts = [oracle.rk_step(om, ref, "rk4") for _ in range(n)]
    np.testing.assert_allclose(dts, odts, rtol=1e-13)
    assert rel_l1(got, ref, sp).max() <= 1e-12


def test_advection_hll_with_a_zero_velocity_component():
    """v_y = 0: the HLL flux through y faces is zero (no wave)."""
    sp, rounds = refined(2, 16, 2, 1, velocity=(1.0, 0.0))
    om, f = make_pair(sp, 0, rounds)
    lev, g = om.blocks()
    u = synth.advection_gaussian(sp, lev, g, R=0.2)
    got, _ = run(f, u.copy(), 8)
    ref = u.copy()
    oracle.run_heun(om, ref, 8)
    assert rel_l1(got, ref, sp).max() <= 1e-12


@pytest.mark.parametrize("ndim,limiter", [(2, 2), (3, 2), (2, 3), (3, 3)])
def test_advection_fp32_matches_oracle(ndim, limiter):
    N = 16
    nt = 8 if ndim == 2 else 2
    sp = synth.advection_spec(ndim=ndim, N=N, ntrees=(nt,) * ndim + (1,) * (3 - ndim), limiter=limiter,
                              velocity=(1.0, 1.0, 1.0), max_level=1)
    om, f = make_pair(sp, 0, [lambda s, lev, g: synth.ball_flags(s, lev, g, (0.5, 0.5, 0.5), (0.2,))],
                      precision=32, n_states=4)
    lev, g = om.blocks()
    u = synth.advection_gaussian(sp, lev, g, R=0.15)
    scheme = "rk4" if limiter == 3 else "heun"
    f.set_state(0, u.astype(np.float32))
    f.compute_dt(0)
    f.step(20, scheme=scheme, use_graph=True, gather=limiter != 3)
    assert f.sync_status() == amr.AMR_OK
    ref = u.copy()
    for _ in range(20):
        oracle.rk_step(om, ref, scheme)
    assert rel_l1(f.get_state(0), ref, sp).max() <= 1e-5


@pytest.mark.parametrize("ndim", [2, 3])
def test_advection_conservation_error_at_rounding(ndim):
    """Sec. 4.1.1 on the GPU: the conservation error of Eq. 18 after many
    steps across refinement boundaries stays at rounding level in FP64."""
    sp, rounds = refined(ndim, 16 if ndim == 2 else 8, 2, 0)
    om, f = make_pair(sp, 0, rounds)
    lev, g = om.blocks()
    u = synth.advection_sphere(sp, lev, g, R=0.2, delta=0.1)
    f.set_state(0, u)
    f.compute_dt(0)
    s0 = f.conserved(0)[0]
    f.step(100 if ndim == 2 else 40, use_graph=True, gather=True)
    assert f.sync_status() == amr.AMR_OK
    s1 = f.conserved(0)[0]
    assert abs(s1 - s0) <= 1e-13 * abs(s0), (s0, s1)
    assert abs(s0 - om.conserved(u)[0]) <= 1e-13 * abs(s0)


def test_advection_flags_bit_exact():
    sp, rounds = refined(2, 16, 2, 0)
    om, f = make_pair(sp, 0, rounds)
    lev, g = om.blocks()
    u = synth.advection_sphere(sp, lev, g, R=0.25, delta=0.1)
    f.set_state(0, u)
    f.fill_ghosts(0)
    ref = u.copy()
    om.fill_ghosts(ref)
    for c_ref, c_deref in ((5e-2, 6.25e-3), (2e-2, 1e-2), (0.3, 0.1)):
        exp = om.lohner_flags(ref, c_ref, c_deref)
        np.testing.assert_array_equal(f.flag(0, c_ref, c_deref), exp)
    exp = om.lohner_flags(ref)
    assert (exp == 1).any() and (exp == -1).any()


def test_advection_refuses_features_and_gravity():
    sp = synth.advection_spec(ndim=2, N=16, ntrees=(2, 2, 1))
    f = amr.Forest(sp, 0, precision=32)
    with pytest.raises(amr.AmrError) as e:
        f.features(0)
    assert e.value.status == amr.AMR_EINVAL
    bad = synth.advection_spec(ndim=2, N=16, ntrees=(2, 2, 1), gravity=(0.0, -1.0, 0.0))
    with pytest.raises(amr.AmrError):
        amr.Forest(bad, 0)


@pytest.mark.parametrize("ndim,N", [(2, 8), (2, 16), (2, 32), (3, 8), (3, 16)])
@pytest.mark.parametrize("limiter", [0, 1, 2])
def test_advection_fp32_block_kernel_matches_oracle(ndim, N, limiter):
    """The FP32 block kernel for advection (MUSCL slopes, gathered halos,
    CUDA graph) on 3-level meshes with flux fixing: relative L1 <= 1e-5
    after 12 Heun steps against the FP64 oracle."""
    nt = (64 if ndim == 2 else 32) // N
    sp = synth.advection_spec(ndim=ndim, N=N, ntrees=(nt,) * ndim + (1,) * (3 - ndim), limiter=limiter,
                              velocity=(1.0, -0.6, 0.8), max_level=2)
    c = (0.62, 0.58, 0.6)
    fl = lambda s, lev, g: synth.ball_flags(s, lev, g, c, (0.2, 0.1))
    om, f = make_pair(sp, 0, [fl, fl], precision=32)
    lev, g = om.blocks()
    assert lev.max() == 2
    u = synth.advection_gaussian(sp, lev, g, R=0.15)
    f.set_state(0, u.astype(np.float32))
    f.compute_dt(0)
    f.step(12, use_graph=True, gather=True)
    assert f.sync_status() == amr.AMR_OK
    ref = u.copy()
    oracle.run_heun(om, ref, 12)
    assert rel_l1(f.get_state(0), ref, sp).max() <= 1e-5


@pytest.mark.parametrize("ndim", [2, 3])
def test_advection_block_kernel_agrees_with_per_cell_kernel(ndim):
    """Launch shapes of the block kernel are bit-identical; the per-cell
    kernel (shape >= 100) agrees within FP32 rounding order."""
    sp = synth.advection_spec(ndim=ndim, N=16, ntrees=(8 if ndim == 2 else 4,) * ndim + (1,) * (3 - ndim), limiter=2)
    f = amr.Forest(sp, 0, precision=32)
    lev, g = f.blocks()
    u = synth.advection_sphere(sp, lev, g, R=0.3, delta=0.1).astype(np.float32)
    res = {}
    for choice in (1, 2, 0, 101):
        f.set_launch_shape(choice)
        f.set_state(0, u)
        f.compute_dt(0)
        f.step(6, use_graph=True, gather=True)
        assert f.sync_status() == amr.AMR_OK
        res[choice] = f.get_state(0)
    for c in (2, 0):
        np.testing.assert_array_equal(res[c], res[1])
    assert rel_l1(res[101], res[1].astype(np.float64), sp).max() <= 1e-6
