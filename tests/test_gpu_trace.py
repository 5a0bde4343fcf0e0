"""Per-phase timing (the timers of Sec. 2.8; the ghost-cell share of the
breakdowns in Sec. 5.2 and 5.4) on the GPU: which phases a step, a regrid
and the reductions record, and that tracing changes no result and no launch
count."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

amr = pytest.importorskip("paper_2605_07612_b300")

from test_gpu_parity import AMR2, SPEC_2D_AMR, ball  # noqa: E402


def amr2d(precision=32, **kw):
    sp = synth.MeshSpec(**dict(SPEC_2D_AMR, **kw))
    f = amr.Forest(sp, 0, max_blocks=1024, precision=precision, n_states=4)
    for fl in AMR2:
        lev, g = f.blocks()
        f.regrid(fl(sp, lev, g))
    lev, g = f.blocks()
    assert lev.max() == 2
    return sp, f, synth.kelvin_helmholtz(sp, lev, g, seed=41).astype(f.dtype)


@pytest.mark.parametrize("gather", [False, True])
def test_traced_steps_record_each_phase_and_match_untraced(gather):
    """3 Heun steps on a 3-level mesh: per stage one ghost round 1 and 2
    record, one stage and one flux-fix record; the dt commit once per step.
    The traced run (which falls back from the graph) is bit-identical to the
    graph replay and issues the same launches."""
    sp, f, u = amr2d()
    res, launches = {}, {}
    for traced in (False, True):
        f.trace(traced)
        f.set_state(0, u)
        f.compute_dt(0)
        f.trace_read()                          # drop the compute_dt record
        l0 = f.launch_count()
        f.step(3, use_graph=True, gather=gather)
        assert f.sync_status() == amr.AMR_OK
        launches[traced] = f.launch_count() - l0
        res[traced] = f.get_state(0)
        t = f.trace_read()
        if not traced:
            assert all(v == (0.0, 0) for v in t.values())
            continue
        for p in ("ghost_r1", "ghost_r2", "stage", "fluxfix"):
            assert t[p][1] == 6 and t[p][0] > 0.0, (p, t[p])
        assert t["dt"][1] == 3
        for p in ("conserved", "flags", "transfer", "mesh_host", "pattern_host"):
            assert t[p][1] == 0, (p, t[p])
    f.trace(False)
    np.testing.assert_array_equal(res[True], res[False])
    assert launches[True] == launches[False]


def test_uniform_gathered_step_has_no_separate_ghost_fill():
    """A periodic uniform mesh with gathered halos: every ghost is read by the
    stage itself, so no ghost round runs."""
    sp = synth.MeshSpec(ndim=3, N=16, ng=2, ntrees=(2, 2, 2))
    f = amr.Forest(sp, 0, precision=32)
    lev, g = f.blocks()
    f.set_state(0, synth.fourier3d(sp, lev, g, seed=3).astype(np.float32))
    f.compute_dt(0)
    f.trace(True)
    f.step(2, gather=True)
    t = f.trace_read()
    assert t["ghost_r1"][1] == 0 and t["ghost_r2"][1] == 0
    assert t["stage"][1] == 4 and t["fluxfix"][1] == 0 and t["dt"][1] == 2
    f.step(1, gather=False)                   # halos from the ghost fill instead
    t = f.trace_read()
    assert t["ghost_r1"][1] == 2 and t["ghost_r2"][1] == 0 and t["stage"][1] == 2


def test_traced_regrid_reductions_and_autotune():
    """A regrid records the flag kernel, the mesh work on the host, the
    pattern build, the transfer and the new time step; conserved sums one
    record; the autotuner none."""
    sp, f, u = amr2d()
    f.set_state(0, u)
    f.trace(True)
    lev, g = f.blocks()
    assert f.regrid(None, c_ref=0.02, c_deref=0.01)
    t = f.trace_read()
    for p in ("ghost_r1", "flags", "mesh_host", "transfer", "pattern_host", "dt"):
        assert t[p][1] == 1, (p, t[p])
    assert t["stage"][1] == 0
    f.conserved(0)
    assert f.trace_read()["conserved"][1] == 1
    f.compute_dt(0)
    f.trace_read()
    f.autotune()
    assert all(v[1] == 0 for v in f.trace_read().values())
    f.trace(False)


def test_traced_weno5_stage():
    """The two passes of a WENO5 stage (face fluxes, update) are one stage
    record."""
    sp = synth.MeshSpec(ndim=2, N=16, ng=3, ntrees=(4, 4, 1), max_level=1, limiter=3)
    f = amr.Forest(sp, 0, max_blocks=256, precision=64)
    lev, g = f.blocks()
    f.regrid(synth.ball_flags(sp, lev, g, (0.5, 0.5), (0.2,)))
    lev, g = f.blocks()
    f.set_state(0, synth.kelvin_helmholtz(sp, lev, g, seed=42))
    f.compute_dt(0)
    f.trace(True)
    f.trace_read()
    f.step(2)
    assert f.sync_status() == amr.AMR_OK
    t = f.trace_read()
    assert t["stage"][1] == 4 and t["ghost_r1"][1] == 4 and t["ghost_r2"][1] == 4 and t["fluxfix"][1] == 4
