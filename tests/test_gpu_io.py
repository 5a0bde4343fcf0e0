"""Checkpoint/restart and XDMF output (Sec. 2.8) on the GPU: a run restarted
from a checkpoint continues bit-identically, and the XDMF files describe
every block with the geometry of its level and hold its interior cells."""
import xml.etree.ElementTree as ET

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

amr = pytest.importorskip("paper_2605_07612_b300")


def ball(centre, radii):
    return lambda sp, lev, g: synth.ball_flags(sp, lev, g, centre, radii)


@pytest.mark.parametrize("precision", [64, 32])
def test_restart_continues_bit_identically(tmp_path, precision):
    sp = synth.MeshSpec(ndim=2, N=16, ng=2, ntrees=(4, 4, 1), max_level=2)
    f = amr.Forest(sp, 0, max_blocks=1024, precision=precision)
    for _ in range(2):
        lev, g = f.blocks()
        f.regrid(synth.ball_flags(sp, lev, g, (0.4, 0.55), (0.3, 0.15)))
    lev, g = f.blocks()
    f.set_state(0, synth.kelvin_helmholtz(sp, lev, g, seed=1).astype(f.dtype))
    f.compute_dt(0)
    f.step(5)
    path = str(tmp_path / "run.ckpt")
    f.save(path)
    g2 = amr.Forest.load(path)
    assert g2.get_dt() == f.get_dt()
    for a, b in zip(f.blocks(), g2.blocks()):
        np.testing.assert_array_equal(a, b)
    f.step(7, use_graph=True)
    g2.step(7, use_graph=True)
    np.testing.assert_array_equal(f.get_state(0), g2.get_state(0))
    assert g2.sync_status() == amr.AMR_OK


def test_restart_of_a_batch(tmp_path):
    specs = [synth.MeshSpec(ndim=2, N=8, ng=2, ntrees=(2, 2, 1), max_level=1),
             synth.MeshSpec(ndim=2, N=8, ng=2, ntrees=(3, 2, 1), max_level=1, cfl=0.3)]
    f = amr.Forest(None, batch=[(specs[0], 1, 64), (specs[1], 0, 64)], precision=64)
    lev, g = f.blocks()
    parts = []
    for i, sp in enumerate(specs):
        first, n = f.instance_blocks(i)
        parts.append(synth.kelvin_helmholtz(sp, lev[first:first + n], g[first:first + n], seed=i))
    f.set_state(0, np.concatenate(parts))
    f.compute_dt(0)
    f.step(3)
    path = str(tmp_path / "batch.ckpt")
    f.save(path)
    g2 = amr.Forest.load(path)
    assert g2.n_instances == 2 and g2.specs[1].cfl == 0.3
    np.testing.assert_array_equal(f.get_dts(), g2.get_dts())
    f.step(4)
    g2.step(4)
    np.testing.assert_array_equal(f.get_state(0), g2.get_state(0))


@pytest.mark.parametrize("ndim", [2, 3])
def test_xdmf_output_describes_blocks_and_data(tmp_path, ndim):
    if ndim == 2:
        sp = synth.MeshSpec(ndim=2, N=8, ng=2, ntrees=(3, 2, 1), max_level=1, lo=(0.5, -1.0, 0.0), length=(3.0, 2.0, 1.0))
    else:
        sp = synth.MeshSpec(ndim=3, N=8, ng=2, ntrees=(2, 2, 2), max_level=1)
    f = amr.Forest(sp, 0, max_blocks=512, precision=32)
    lev, g = f.blocks()
    f.regrid(synth.point_flags(sp, lev, g, (0.6,) * ndim, sp.max_level))
    lev, g = f.blocks()
    u = (synth.kelvin_helmholtz(sp, lev, g) if ndim == 2 else synth.fourier3d(sp, lev, g)).astype(np.float32)
    f.set_state(0, u)
    base = str(tmp_path / "out")
    f.write_xdmf(0, base)
    root = ET.parse(base + ".xmf").getroot()
    grids = root.findall("./Domain/Grid/Grid")
    assert len(grids) == f.n
    raw = np.fromfile(base + ".bin", dtype=np.float32)
    N, V = sp.N, sp.nvar
    assert raw.size == f.n * V * N ** ndim
    sl = tuple(slice(sp.ng, sp.ng + N) for _ in range(ndim))
    for b, gr in enumerate(grids):
        dims = [int(x) for x in gr.find("Topology").get("Dimensions").split()]
        assert dims == [N + 1] * ndim
        org, dx = [np.array([float(x) for x in d.text.split()])[::-1] for d in gr.find("Geometry").findall("DataItem")]
        h = np.array([sp.length[d] / sp.ntrees[d] / (N << lev[b]) for d in range(ndim)])
        np.testing.assert_allclose(dx, h, rtol=1e-15)
        np.testing.assert_allclose(org, [sp.lo[d] + g[b, d] * N * h[d] for d in range(ndim)], rtol=1e-15, atol=1e-15)
        atts = gr.findall("Attribute")
        assert [a.get("Name") for a in atts] == (["rho", "mx", "my", "E"] if ndim == 2 else ["rho", "mx", "my", "mz", "E"])
        for v, a in enumerate(atts):
            item = a.find("DataItem")
            off = int(item.get("Seek")) // 4
            got = raw[off:off + N ** ndim].reshape((N,) * ndim)
            want = u[b, v].reshape((sp.side,) * ndim)[sl]
            np.testing.assert_array_equal(got, want)
