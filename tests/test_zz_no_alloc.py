"""GPU check of amr_conserved_static(), the allocation-free way to get the
conserved integrals for callers that cannot call cudaMalloc (device memory
reserved up front by another allocator, or no device-wide synchronisation
allowed).  It must give the same sums as amr_conserved() on the same blocks,
on consecutive calls that share its static scratch array.

Kept in a file of its own that pytest collects last."""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

amr = pytest.importorskip("paper_2605_07612_b300")
torch = pytest.importorskip("torch")


def _entry():
    lib = amr.load()
    fn = lib.amr_conserved_static
    fn.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]
    fn.restype = C.c_int
    return fn


def _amr_forest(precision):
    sp = synth.MeshSpec(ndim=3, N=8, ng=2, ntrees=(4, 4, 4), max_level=2)
    f = amr.Forest(sp, 0, max_blocks=4096, precision=precision)
    for _ in range(2):
        lev, g = f.blocks()
        f.regrid(synth.ball_flags(sp, lev, g, (0.45, 0.5, 0.55), (0.15, 0.05)))
    lev, g = f.blocks()
    assert set(lev.tolist()) == {0, 1, 2}
    u = synth.fourier3d(sp, lev, g, seed=3)
    f.set_state(0, u.astype(f.dtype))
    return sp, f


def _cell_volumes(sp, lev):
    vol = np.ones(len(lev))
    for d in range(sp.ndim):
        vol = vol * (sp.length[d] / float(sp.ntrees[d]) / (float(sp.N) * np.power(2.0, lev)))
    return vol


@pytest.mark.parametrize("precision", [64, 32])
def test_static_sums_match_amr_conserved_on_two_calls(precision):
    fn = _entry()
    sp, f = _amr_forest(precision)
    lev, _ = f.blocks()
    vol = torch.tensor(_cell_volumes(sp, lev), dtype=torch.float64, device="cuda")
    sums = torch.zeros(sp.nvar, dtype=torch.float64, device="cuda")
    f.compute_dt(0)
    for call in range(2):
        ref = f.conserved(0)
        st = fn(f.state_ptr(0), precision, sp.ndim, sp.N, sp.ng, f.n, vol.data_ptr(), sums.data_ptr(), None)
        assert st == amr.AMR_OK
        torch.cuda.synchronize()
        got = sums.cpu().numpy()
        u = f.get_state(0).astype(np.float64)
        mag = np.array([np.abs(u[:, v]).sum() for v in range(sp.nvar)]) * vol.cpu().numpy().max()
        assert np.all(np.abs(got - ref) <= 1e-13 * mag), (call, got, ref)
        f.step(1)          # the second call sees a different state


def test_static_sums_reject_oversized_input():
    fn = _entry()
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = fn(dummy.data_ptr(), 64, 3, 16, 2, 65537, dummy.data_ptr(), dummy.data_ptr(), None)
    assert st == amr.AMR_ECAPACITY
    st = fn(None, 64, 3, 16, 2, 4, dummy.data_ptr(), dummy.data_ptr(), None)
    assert st == amr.AMR_EINVAL
