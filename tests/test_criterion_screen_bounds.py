"""Host check of the error bounds behind the criterion's FP32 screen.

The GPU decides a block's refinement flag in FP32 when an interval around
its largest criterion value (Eq. 12) lies clear of both thresholds, and
leaves the block to the FP64 evaluation otherwise.  That is exact only if
the interval always holds the FP64 value.  Here the screen's arithmetic is
modelled in numpy FP32 -- every operation rounded on its own (the GPU's
fused multiply-adds only round less), each approximate reciprocal off by up
to one unit in the last place in a random direction -- on random stencils
with densities over six decades, speeds up to Mach 30 and near-cancelling
pressures, and the FP64 value of each 1D indicator must lie inside the
modelled interval whenever the screen would keep the stencil.
"""
import numpy as np
import pytest

F = np.float32


def rcp(x, rng):
    """1/x in FP32 with an error of up to one unit in the last place."""
    r = (F(1.0) / x).astype(F)
    return (r * (F(1.0) + rng.choice([-1.0, 0.0, 1.0], size=r.shape).astype(F) * F(2.0 ** -23))).astype(F)


def primitives_fp32(U, gm1, wide, rng):
    """Density, pressure and the pressure bound as the screen computes them."""
    rho = U[0]
    r = rcp(rho, rng)
    ke = np.zeros_like(rho)
    for d in range(3):
        w = (U[1 + d] * r).astype(F)
        ke = (ke + (w * w).astype(F)).astype(F)
    ke = ((F(0.5) * rho).astype(F) * ke).astype(F)
    p = (F(gm1) * (U[4] - ke).astype(F)).astype(F)
    kp = F(2.0 ** -17) if wide else F(2.0 ** -18)
    bp = (kp * (F(gm1) * ke + np.abs(p)).astype(F) + F(1e-30)).astype(F)
    return rho, p, bp


def interval(am, a0, ap, bm, b0, bq, eps, eps_abs, rng):
    num = np.abs((am - (F(2.0) * a0)).astype(F) + ap).astype(F)
    ustar = ((np.abs(am) + F(2.0) * np.abs(a0)).astype(F) + np.abs(ap)).astype(F)
    den = (((F(eps_abs) + np.abs(a0 - am)).astype(F) + np.abs(ap - a0)).astype(F) + (F(eps) * ustar).astype(F)).astype(F)
    B = (bm + F(2.0) * b0 + bq).astype(F)
    Bn = (B + F(2.0 ** -21) * ustar).astype(F)
    Bd = ((F(1.0) + F(eps)) * B + F(2.0 ** -20) * den).astype(F)
    keep = den > F(2.0) * Bd
    with np.errstate(divide="ignore", invalid="ignore"):
        hi = ((num + Bn) * rcp((den - Bd).astype(F), rng)).astype(F) * F(1.0 + 2.0 ** -19)
        lo = (np.maximum(num - Bn, F(0.0)) * rcp((den + Bd).astype(F), rng)).astype(F) * F(1.0 - 2.0 ** -19)
    return lo.astype(F), hi.astype(F), keep


def lohner_fp64(um, u0, up, eps, eps_abs):
    num = np.abs(um - 2.0 * u0 + up)
    ustar = np.abs(um) + 2.0 * np.abs(u0) + np.abs(up)
    den = eps_abs + np.abs(u0 - um) + np.abs(up - u0) + eps * ustar
    return num / den


def random_states(rng, n, cancel):
    rho = np.exp(rng.uniform(np.log(1e-3), np.log(1e3), n))
    p = np.exp(rng.uniform(np.log(1e-3), np.log(1e3), n))
    c = np.sqrt(1.4 * p / rho)
    mach = rng.uniform(0.0, 30.0, n) if cancel else rng.uniform(0.0, 2.0, n)
    dirs = rng.normal(size=(3, n))
    dirs /= np.linalg.norm(dirs, axis=0)
    v = dirs * mach * c
    E = p / 0.4 + 0.5 * rho * (v * v).sum(axis=0)
    return np.stack([rho, rho * v[0], rho * v[1], rho * v[2], E])


@pytest.mark.parametrize("wide", [False, True])
@pytest.mark.parametrize("cancel", [False, True])
def test_fp32_interval_holds_the_fp64_indicator(wide, cancel):
    rng = np.random.default_rng(11 + 2 * int(wide) + int(cancel))
    n = 200_000
    eps, eps_abs, gm1 = 1e-2, 1e-10, 0.4
    # stencils of three neighbouring cells: the middle one plus small to large
    # relative jumps, so that the indicator spans smooth and shocked values
    mid = random_states(rng, n, cancel)
    jumps = np.exp(rng.uniform(np.log(1e-7), np.log(1.0), (2, n)))
    cells = []
    for s in (-1.0, 1.0):
        k = 0 if s < 0 else 1
        scale = 1.0 + s * jumps[k] * rng.uniform(-1.0, 1.0, n)
        u = mid * scale
        u[4] = np.maximum(u[4], 0.5 * (u[1] ** 2 + u[2] ** 2 + u[3] ** 2) / u[0] * (1.0 + 1e-7))   # p > 0
        cells.append(u)
    um, u0, up = cells[0], mid, cells[1]
    # the state's own numbers: FP32 values (an FP32 state) or FP64 values
    # that the screen rounds to FP32 (an FP64 state)
    if wide:
        src = [x for x in (um, u0, up)]
    else:
        src = [x.astype(F).astype(np.float64) for x in (um, u0, up)]
    U32 = [x.astype(F) for x in src]
    prim32 = [primitives_fp32(x, gm1, wide, rng) for x in U32]
    for which in (0, 1):
        if which == 0:
            a = [q[0] for q in prim32]
            kr = F(2.0 ** -23) if wide else F(0.0)
            b = [(kr * x).astype(F) for x in a]
        else:
            a = [q[1] for q in prim32]
            b = [q[2] for q in prim32]
        lo, hi, keep = interval(a[0], a[1], a[2], b[0], b[1], b[2], eps, eps_abs, rng)
        # the FP64 evaluation of the same state (the value k_flags compares)
        def prim64(U):
            rho = U[0]
            ke = sum((U[1 + d] / rho) ** 2 for d in range(3)) * (0.5 * rho)
            return rho if which == 0 else gm1 * (U[4] - ke)
        e64 = lohner_fp64(prim64(src[0]), prim64(src[1]), prim64(src[2]), eps, eps_abs)
        ok = keep & np.isfinite(hi)
        assert ok.mean() > 0.9
        inside = (lo.astype(np.float64) <= e64) & (e64 <= hi.astype(np.float64))
        assert np.all(inside[ok]), (which, np.flatnonzero(ok & ~inside)[:5])
