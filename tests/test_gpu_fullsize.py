"""Parity at the benchmark's full size and launch configuration: the uniform
periodic 256^3 mesh of 16^3 blocks in FP32, same-level halos gathered by the
stage kernel, one step replayed as a CUDA graph, launch shape chosen by the
autotuner.  20 Heun steps are compared with the FP64 oracle run on the whole
mesh; conservation of the FP64 integrals is checked over 20 steps for 8^3,
16^3 and 32^3 blocks."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

amr = pytest.importorskip("paper_2605_07612_b300")


def spec_of(n):
    nt = 256 // n
    return synth.MeshSpec(ndim=3, N=n, ng=2, ntrees=(nt, nt, nt))


def test_full_size_20_steps_match_oracle():
    """The headline configuration for 20 Heun steps (FP32 GPU, FP64 oracle
    on the host cores)."""
    sp = spec_of(16)
    f = amr.Forest(sp, 0, precision=32)
    lev, g = f.blocks()
    u = synth.fourier3d(sp, lev, g, seed=1)
    f.set_state(0, u.astype(np.float32))
    f.compute_dt(0)
    f.autotune()
    f.step(20, use_graph=True, gather=True)
    assert f.sync_status() == amr.AMR_OK
    got = f.get_state(0)
    m = oracle.Mesh(sp, 0)
    oracle.run_heun(m, u, 20)
    del m
    sl = slice(sp.ng, sp.ng + sp.N)
    for v in range(sp.nvar):
        a = got[:, v].reshape(-1, sp.side, sp.side, sp.side)[:, sl, sl, sl].astype(np.float64)
        b = u[:, v].reshape(-1, sp.side, sp.side, sp.side)[:, sl, sl, sl]
        err = np.abs(a - b).sum() / np.abs(b).sum()
        assert err <= 1e-5, (v, err)


@pytest.mark.parametrize("n", [8, 16, 32])
def test_full_size_conservation(n):
    sp = spec_of(n)
    f = amr.Forest(sp, 0, precision=32)
    lev, g = f.blocks()
    u = synth.fourier3d(sp, lev, g, seed=2).astype(np.float32)
    f.set_state(0, u)
    s0 = f.conserved(0)
    scale = np.array([np.abs(u[:, v].astype(np.float64)).sum() for v in range(sp.nvar)]) / f.n / sp.N ** 3
    f.compute_dt(0)
    f.autotune()
    f.step(20, use_graph=True, gather=True)
    assert f.sync_status() == amr.AMR_OK
    drift = np.abs(f.conserved(0) - s0) / scale
    assert drift.max() < 2e-6, drift
