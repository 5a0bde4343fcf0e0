"""Host-side checks of the CUDA library (no GPU needed): the shared object
loads and exports every function include/amr.h declares; configurations are
validated; the production forest and face-walk ghost pattern builder agree
bit for bit with the oracle's brute-force classification (Sec. 2.2, 2.6)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
import synth
import paper_2605_07612_b300 as amr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "amr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(amr_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = amr.load()
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(names) == sorted(amr.EXPORTED)


def test_invalid_configs_are_rejected():
    lib = amr.load()
    sp = synth.MeshSpec(ndim=3, N=16, ng=2, ntrees=(2, 2, 2), max_level=1)
    h = C.c_void_p()
    for field, value in [("block_n", 12), ("n_ghost", 9), ("n_var", 4), ("precision", 16), ("ndim", 4),
                         ("max_level", 40), ("max_blocks", 0)]:
        cfg = amr.config_from_spec(sp, 64, host_only=True)
        setattr(cfg, field, value)
        assert lib.amr_create_forest(C.byref(cfg), 0, C.byref(h)) == amr.AMR_EINVAL, field
    cfg = amr.config_from_spec(sp, 64, host_only=True)
    cfg.periodic[0] = 0            # non-periodic x without a boundary kind
    assert lib.amr_create_forest(C.byref(cfg), 0, C.byref(h)) == amr.AMR_EINVAL
    cfg = amr.config_from_spec(sp, 7, host_only=True)    # 8 blocks at level 0
    assert lib.amr_create_forest(C.byref(cfg), 0, C.byref(h)) == amr.AMR_ECAPACITY
    assert lib.amr_create_forest(None, 0, C.byref(h)) == amr.AMR_EINVAL


def test_host_only_forest_refuses_block_data():
    sp = synth.MeshSpec(ndim=2, N=8, ng=2, ntrees=(2, 2, 1), max_level=1)
    f = amr.Forest(sp, 0, max_blocks=16, host_only=True)
    with pytest.raises(amr.AmrError) as e:
        f.fill_ghosts(0)
    assert e.value.status == amr.AMR_ESTATE
    with pytest.raises(amr.AmrError) as e:
        f.regrid(None)
    assert e.value.status == amr.AMR_ESTATE


def test_capacity_overflow_leaves_mesh_unchanged():
    sp = synth.MeshSpec(ndim=2, N=8, ng=2, ntrees=(2, 2, 1), max_level=2)
    f = amr.Forest(sp, 0, max_blocks=8, host_only=True)
    pat0 = f.pattern().copy()
    with pytest.raises(amr.AmrError) as e:
        f.regrid(np.ones(4, dtype=np.int8))      # 16 blocks > 8
    assert e.value.status == amr.AMR_ECAPACITY
    assert f.n == 4
    np.testing.assert_array_equal(f.pattern(), pat0)


def random_pair(ndim, seed, rounds=3, diagonal=0):
    rng = np.random.default_rng(1000 + seed)
    if ndim == 2:
        nt = (int(rng.integers(1, 5)), int(rng.integers(1, 5)), 1)
        per = (int(rng.integers(2)), int(rng.integers(2)), 1)
        sp = synth.MeshSpec(ndim=2, N=8, ng=2, ntrees=nt, periodic=per, max_level=3,
                            bc_type=(1, 1, 2, 2, 0, 0))
    else:
        nt = tuple(int(x) for x in rng.integers(1, 4, 3))
        per = tuple(int(x) for x in rng.integers(0, 2, 3))
        sp = synth.MeshSpec(ndim=3, N=8, ng=2, ntrees=nt, periodic=per, max_level=3,
                            bc_type=(1, 2, 1, 2, 3, 3))
    sp.diagonal_ghosts = diagonal
    lvl0 = int(rng.integers(0, 2))
    om = oracle.Mesh(sp, lvl0)
    pm = amr.Forest(sp, lvl0, max_blocks=200000, host_only=True)
    for _ in range(rounds):
        flags = rng.choice(np.array([-1, 0, 1], dtype=np.int8), size=om.n, p=[0.3, 0.45, 0.25])
        om = om.adapt(flags)
        pm.regrid(flags)
    return sp, om, pm


@pytest.mark.parametrize("seed", range(60))
def test_production_pattern_matches_brute_force_2d(seed):
    sp, om, pm = random_pair(2, seed)
    lo, go = om.blocks()
    lp, gp = pm.blocks()
    np.testing.assert_array_equal(lo, lp)
    np.testing.assert_array_equal(go, gp)
    np.testing.assert_array_equal(om.pattern(), pm.pattern())


@pytest.mark.parametrize("seed", range(25))
def test_production_pattern_matches_brute_force_3d(seed):
    sp, om, pm = random_pair(3, seed)
    lo, go = om.blocks()
    lp, gp = pm.blocks()
    np.testing.assert_array_equal(lo, lp)
    np.testing.assert_array_equal(go, gp)
    np.testing.assert_array_equal(om.pattern(), pm.pattern())


@pytest.mark.parametrize("ndim,seed", [(2, s) for s in range(20)] + [(3, s) for s in range(10)])
def test_production_pattern_with_diagonal_ghosts_matches_brute_force(ndim, seed):
    """With edge/corner ghosts switched on, the production pattern (face walk
    plus same-level diagonal neighbours) equals the oracle's point-location
    brute force, entry for entry."""
    sp, om, pm = random_pair(ndim, seed, diagonal=1)
    po, pp = om.pattern(), pm.pattern()
    np.testing.assert_array_equal(po, pp)
    assert (pp[:, 0] == 4).any()


def test_uniform_3d_configs_shape():
    """The 256^3 uniform meshes of the benchmark: 16^3 blocks -> 4096 blocks, 6 SRL faces each."""
    for n, nt in ((8, 32), (16, 16), (32, 8)):
        sp = synth.MeshSpec(ndim=3, N=n, ng=2, ntrees=(nt, nt, nt), max_level=0)
        f = amr.Forest(sp, 0, host_only=True)
        assert f.n == nt ** 3
        pat = f.pattern()
        assert len(pat) == 6 * nt ** 3 and np.all(pat[:, 0] == amr.KIND_SRL)


def test_batch_pattern_is_union_of_instance_patterns():
    """A forest of several independent instances numbers their blocks
    consecutively; its pattern is every instance's pattern with block
    indices shifted, in canonical order, and BC rows renumbered."""
    specs = [synth.MeshSpec(ndim=2, N=8, ng=2, ntrees=(2, 3, 1), max_level=2),
             synth.MeshSpec(ndim=2, N=8, ng=2, ntrees=(4, 1, 1), periodic=(0, 1, 1), max_level=1,
                            bc_type=(2, 2, 0, 0, 0, 0)),
             synth.MeshSpec(ndim=2, N=8, ng=2, ntrees=(1, 1, 1), periodic=(0, 0, 1), max_level=3,
                            bc_type=(1, 1, 1, 1, 0, 0))]
    levels = [1, 0, 2]
    f = amr.Forest(None, batch=[(sp, lv, 4096) for sp, lv in zip(specs, levels)], host_only=True)
    rng = np.random.default_rng(3)
    oms = [oracle.Mesh(sp, lv) for sp, lv in zip(specs, levels)]
    for _ in range(2):
        flags = [rng.choice(np.array([-1, 0, 1], dtype=np.int8), size=m.n) for m in oms]
        oms = [m.adapt(fl) for m, fl in zip(oms, flags)]
        f.regrid(np.concatenate(flags))
    rows, off = [], 0
    for i, m in enumerate(oms):
        first, n = f.instance_blocks(i)
        assert first == off and n == m.n
        pat = m.pattern().astype(np.int64)
        pat[:, 2] += off
        pat[:, 3] = np.where(pat[:, 3] >= 0, pat[:, 3] + off, -1)
        rows.append(pat)
        off += m.n
    exp = np.concatenate(rows)
    exp = exp[np.lexsort((exp[:, 4], exp[:, 2], exp[:, 1], exp[:, 0]))]
    bc = exp[:, 0] == oracle.KIND_BC
    exp[bc, 5] = np.arange(bc.sum())
    np.testing.assert_array_equal(f.pattern(), exp)
    assert f.n_instances == 3


def test_checkpoint_round_trip_host_only(tmp_path):
    """amr_save / amr_load of a host-only forest: the same blocks and ghost
    pattern come back; foreign, truncated and mesh-only files are refused."""
    sp = synth.MeshSpec(ndim=3, N=8, ng=2, ntrees=(3, 2, 2), periodic=(1, 0, 1), max_level=2,
                        bc_type=(0, 0, 2, 2, 0, 0))
    f = amr.Forest(sp, 0, max_blocks=4000, host_only=True)
    rng = np.random.default_rng(3)
    for _ in range(3):
        f.regrid(rng.choice(np.array([-1, 0, 1], dtype=np.int8), size=f.n, p=[0.2, 0.4, 0.4]))
    path = tmp_path / "mesh.ckpt"
    f.save(str(path))
    g = amr.Forest.load(str(path), host_only=True)
    for a, b in zip(f.blocks(), g.blocks()):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(f.pattern(), g.pattern())
    assert g.spec.ntrees == sp.ntrees and g.spec.bc_type == sp.bc_type and g.spec.max_level == 2
    data = path.read_bytes()
    (tmp_path / "bad").write_bytes(b"NOTACKPT" + data[8:])
    (tmp_path / "short").write_bytes(data[: len(data) // 2])
    for name in ("bad", "short"):
        with pytest.raises(amr.AmrError):
            amr.Forest.load(str(tmp_path / name), host_only=True)
    with pytest.raises(amr.AmrError):       # a mesh-only checkpoint has no state for the device
        amr.Forest.load(str(path))


def test_bench_entry_points_exist():
    """The functions the bench's command line dispatches to (the profiles in
    the repository name those command lines) are defined."""
    import bench
    for name in ("run_ours", "run_reference", "run_amr_static", "run_adaptive", "run_ncu_case", "oracle_sample",
                 "ghost_case_spec", "workload_spec", "stage_kernel_hash", "traffic_from_profile", "run_advection"):
        assert callable(getattr(bench, name)), name


def test_advection_config_validation_and_checkpoint(tmp_path):
    """Scalar advection forests: one variable, no gravity, finite velocity;
    the physics and the velocity survive a checkpoint round trip."""
    lib = amr.load()
    h = C.c_void_p()
    sp = synth.advection_spec(ndim=3, N=8, ntrees=(2, 2, 2), velocity=(1.0, -0.5, 0.25), max_level=1)
    for field, value in [("n_var", 5), ("physics", 2)]:
        cfg = amr.config_from_spec(sp, 64, host_only=True)
        setattr(cfg, field, value)
        assert lib.amr_create_forest(C.byref(cfg), 0, C.byref(h)) == amr.AMR_EINVAL, field
    cfg = amr.config_from_spec(sp, 64, host_only=True)
    cfg.gravity[2] = -1.0
    assert lib.amr_create_forest(C.byref(cfg), 0, C.byref(h)) == amr.AMR_EINVAL
    cfg = amr.config_from_spec(sp, 64, host_only=True)
    cfg.velocity[0] = float("nan")
    assert lib.amr_create_forest(C.byref(cfg), 0, C.byref(h)) == amr.AMR_EINVAL
    euler = synth.MeshSpec(ndim=3, N=8, ng=2, ntrees=(2, 2, 2))
    cfg = amr.config_from_spec(euler, 64, host_only=True)
    cfg.n_var = 1
    assert lib.amr_create_forest(C.byref(cfg), 0, C.byref(h)) == amr.AMR_EINVAL
    f = amr.Forest(sp, 0, max_blocks=512, host_only=True)
    f.regrid(synth.ball_flags(sp, *f.blocks(), (0.3, 0.3, 0.3), (0.2,)))
    path = tmp_path / "adv.ckpt"
    f.save(str(path))
    g = amr.Forest.load(str(path), host_only=True)
    assert g.spec.physics == 1 and tuple(g.spec.velocity) == (1.0, -0.5, 0.25) and g.spec.nvar == 1
    np.testing.assert_array_equal(f.pattern(), g.pattern())


def test_trace_times_host_phases_of_a_regrid():
    """Per-phase timing on a host-only forest: a regrid adds one mesh-host
    record and one pattern-build record; nothing is recorded while tracing is
    off, and reading with reset clears the totals."""
    sp = synth.MeshSpec(ndim=2, N=8, ng=2, ntrees=(4, 4, 1), max_level=2)
    f = amr.Forest(sp, 0, max_blocks=1024, host_only=True)
    flags = np.zeros(f.n, dtype=np.int8)
    flags[:3] = 1
    f.regrid(flags)                               # untraced
    t = f.trace_read()
    assert set(t) == set(amr.PHASES) and all(v == (0.0, 0) for v in t.values())
    f.trace(True)
    flags = np.zeros(f.n, dtype=np.int8)
    flags[-2:] = 1
    assert f.regrid(flags)
    t = f.trace_read(reset=False)
    assert t["mesh_host"][1] == 1 and t["pattern_host"][1] == 1
    assert t["mesh_host"][0] >= 0.0 and t["pattern_host"][0] > 0.0
    assert all(t[p][1] == 0 for p in amr.PHASES if not p.endswith("_host"))
    f.trace(False)
    flags = np.zeros(f.n, dtype=np.int8)
    flags[0] = 1
    f.regrid(flags)
    assert f.trace_read() == t                    # off: unchanged; read and reset
    assert all(v == (0.0, 0) for v in f.trace_read().values())


def test_trace_batched_regrid_records_one_host_phase_per_call():
    """A regrid of a batch of two host-only meshes adapts both instances in
    one mesh-host record and rebuilds the pattern once; a regrid that
    changes nothing records the mesh work but no pattern build; a NULL
    handle is refused."""
    sp = synth.MeshSpec(ndim=2, N=8, ng=2, ntrees=(2, 2, 1), max_level=2)
    f = amr.Forest(None, batch=[(sp, 0, 64), (sp, 1, 64)], host_only=True)
    f.trace(True)
    flags = np.zeros(f.n, dtype=np.int8)
    flags[0] = 1
    flags[-1] = 1
    assert f.regrid(flags)
    t = f.trace_read()
    assert t["mesh_host"][1] == 1 and t["pattern_host"][1] == 1
    assert not f.regrid(np.zeros(f.n, dtype=np.int8))
    t = f.trace_read()
    assert t["mesh_host"][1] == 1 and t["pattern_host"][1] == 0
    lib = f.lib
    assert lib.amr_trace(None, 1) == amr.AMR_EINVAL
    assert lib.amr_trace_read(None, None, None, 0) == amr.AMR_EINVAL
