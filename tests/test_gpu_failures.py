"""Failure handling without any GPU fault: device allocations made through the
caller's allocation hook are failed on purpose, on the host.

Every call must then return AMR_ENOMEM (never abort), hand back every byte it
took, and leave the forest usable: a regrid whose allocation fails keeps the
mesh and data it had (or, when only the pattern upload after the transfer
failed, is completed by the next call that needs the pattern)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

amr = pytest.importorskip("paper_2605_07612_b300")
torch = pytest.importorskip("torch")

from test_gpu_parity import ball  # noqa: E402


class Injector:
    """Allocation hook on torch's caching allocator that fails the calls
    numbered fail_from and later (1-based) while armed."""

    def __init__(self, fail_from=None):
        self.calls = 0
        self.fail_from = fail_from
        self.live = {}
        self.alloc = amr.AllocFn(self._alloc)
        self.free = amr.FreeFn(self._free)

    def _alloc(self, size, ctx):
        self.calls += 1
        if self.fail_from is not None and self.calls >= self.fail_from:
            return None
        p = torch.cuda.caching_allocator_alloc(int(size))
        self.live[p] = int(size)
        return p

    def _free(self, p, ctx):
        if p in self.live:
            del self.live[p]
            torch.cuda.caching_allocator_delete(p)

    def config(self, spec, max_blocks, precision=32):
        c = amr.config_from_spec(spec, max_blocks, 2, precision)
        c.dev_alloc = self.alloc
        c.dev_free = self.free
        return c


SPEC = dict(ndim=2, N=16, ng=2, ntrees=(4, 4, 1), max_level=2)


def test_creation_fails_cleanly_at_every_allocation():
    """Failing the k-th device allocation of forest creation, for every k:
    AMR_ENOMEM and nothing left allocated; past the last one, a working
    forest."""
    sp = synth.MeshSpec(**SPEC)
    probe = Injector()
    f = amr.Forest(sp, 0, config=probe.config(sp, 256))
    n_alloc = probe.calls
    f.close()
    assert n_alloc >= 3 and not probe.live
    for k in range(1, n_alloc + 1):
        inj = Injector(fail_from=k)
        with pytest.raises(amr.AmrError) as e:
            amr.Forest(sp, 0, config=inj.config(sp, 256))
        assert e.value.status == amr.AMR_ENOMEM, k
        assert not inj.live, (k, inj.live)


def interior(sp, u):
    S, sl = sp.side, slice(sp.ng, sp.ng + sp.N)
    return u.reshape((u.shape[0], sp.nvar) + (S,) * sp.ndim)[(slice(None), slice(None)) + (sl,) * sp.ndim]


def test_failed_regrid_keeps_mesh_and_data():
    """A regrid whose device allocations fail returns AMR_ENOMEM. Either it
    was refused before the mesh changed (same blocks, same interior data,
    and a retry succeeds) or only the pattern upload after the transfer failed
    (the next call that needs the pattern completes it). In both cases the
    forest then holds the same blocks and interior data as a forest whose
    regrid succeeded at once, and steps bit-identically to it."""
    sp = synth.MeshSpec(**SPEC)
    inj = Injector()
    f = amr.Forest(sp, 0, config=inj.config(sp, 256, precision=64))
    ref = amr.Forest(sp, 0, max_blocks=256, precision=64)
    lev0, g0 = f.blocks()
    u = synth.kelvin_helmholtz(sp, lev0, g0, seed=31)
    fl = ball((0.4, 0.55), (0.3, 0.15))(sp, lev0, g0)
    for h in (f, ref):
        h.set_state(0, u)
    ref.regrid(fl)
    inj.fail_from = inj.calls + 1           # every later allocation fails
    with pytest.raises(amr.AmrError) as e:
        f.regrid(fl)
    assert e.value.status == amr.AMR_ENOMEM
    inj.fail_from = None
    lev, g = f.blocks()
    if len(lev) == len(lev0) and np.array_equal(lev, lev0):
        # the interior as it was (the regrid's ghost fill may have run)
        np.testing.assert_array_equal(interior(sp, f.get_state(0)), interior(sp, u))
        f.regrid(fl)
    else:
        f.fill_ghosts(0)                    # uploads the pattern of the new mesh
    for a, b in zip(f.blocks(), ref.blocks()):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(interior(sp, f.get_state(0)), interior(sp, ref.get_state(0)))
    for h in (f, ref):
        h.compute_dt(0)
        h.step(2)
        assert h.sync_status() == amr.AMR_OK
    np.testing.assert_array_equal(interior(sp, f.get_state(0)), interior(sp, ref.get_state(0)))
    f.close()
    assert not inj.live


def test_weno5_scratch_is_returned():
    """The WENO5 stage's scratch (primitives and face fluxes of every block),
    allocated on first use, goes back through the hook when the forest is
    destroyed."""
    sp = synth.MeshSpec(ndim=2, N=16, ng=3, ntrees=(4, 4, 1), limiter=3)
    inj = Injector()
    f = amr.Forest(sp, 0, config=inj.config(sp, 64, precision=64))
    n0 = len(inj.live)
    lev, g = f.blocks()
    f.set_state(0, synth.kelvin_helmholtz(sp, lev, g, seed=43))
    f.compute_dt(0)
    f.step(1)
    assert f.sync_status() == amr.AMR_OK
    assert len(inj.live) > n0
    f.close()
    assert not inj.live
