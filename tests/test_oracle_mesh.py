"""Pins of the oracle's forest and ghost-pattern classification (Sec. 2.2,
Sec. 2.6) against hand enumeration, closed forms and independent geometry.
CPU only."""
import itertools
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_table(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].strip()
        if line:
            rows.append([int(x) for x in line.split()])
    return np.array(rows, dtype=np.int32)


def spec2(**kw):
    base = dict(ndim=2, N=4, ng=1, ntrees=(2, 1, 1), periodic=(0, 0, 1), max_level=2)
    base.update(kw)
    return synth.MeshSpec(**base)


def test_hand_enumerated_pattern_2d():
    """Golden: a 2x1 brick with tree 0 refined once (derivation in the file)."""
    m = oracle.Mesh(spec2(), 0)
    m2 = m.adapt(np.array([1, 0], dtype=np.int8))
    lev, g = m2.blocks()
    assert lev.tolist() == [1, 1, 1, 1, 0]
    assert g[:, :2].tolist() == [[0, 0], [1, 0], [0, 1], [1, 1], [1, 0]]
    np.testing.assert_array_equal(m2.pattern(), load_table("pattern_2d_brick2x1.txt"))


def test_hand_enumerated_refinement_faces_3d():
    """2x1x1 brick, tree 0 refined: the root of tree 1 receives restriction
    from the four level-1 blocks with x=1, at offsets (y bit, z bit)."""
    sp = synth.MeshSpec(ndim=3, N=4, ng=1, ntrees=(2, 1, 1), periodic=(0, 0, 0), max_level=1)
    m = oracle.Mesh(sp, 0).adapt(np.array([1, 0], dtype=np.int8))
    lev, g = m.blocks()
    assert lev.tolist() == [1] * 8 + [0]
    # Morton order inside tree 0, x lowest bit
    assert g[:8].tolist() == [[x, y, z] for z in (0, 1) for y in (0, 1) for x in (0, 1)]
    pat = m.pattern()
    f2c = pat[pat[:, 0] == oracle.KIND_F2C]
    assert f2c[:, 1:5].tolist() == [[0, 8, 1, 0], [0, 8, 3, 1], [0, 8, 5, 2], [0, 8, 7, 3]]
    c2f = pat[pat[:, 0] == oracle.KIND_C2F]
    assert c2f[:, 1:5].tolist() == [[1, 1, 8, 0], [1, 3, 8, 1], [1, 5, 8, 2], [1, 7, 8, 3]]


def morton_decode(n, ndim, bits):
    c = [0, 0, 0]
    for b in range(bits):
        for d in range(ndim):
            c[d] |= ((n >> (ndim * b + d)) & 1) << b
    return c


@pytest.mark.parametrize("ndim,ntrees,level", [(2, (3, 2, 1), 3), (3, (2, 1, 2), 2)])
def test_leaf_order_closed_form(ndim, ntrees, level):
    """Uniform forest: block n = tree-major (row-major trees), Morton inside."""
    sp = synth.MeshSpec(ndim=ndim, N=4, ng=1, ntrees=ntrees, max_level=level)
    lev, g = oracle.Mesh(sp, level).blocks()
    per_tree = 1 << (ndim * level)
    for n in range(len(lev)):
        t, mo = divmod(n, per_tree)
        tx = t % ntrees[0]
        ty = (t // ntrees[0]) % ntrees[1]
        tz = t // (ntrees[0] * ntrees[1])
        loc = morton_decode(mo, ndim, level)
        exp = [tx * (1 << level) + loc[0], ty * (1 << level) + loc[1], (tz * (1 << level) + loc[2]) if ndim == 3 else 0]
        assert g[n].tolist() == exp


@pytest.mark.parametrize("ndim", [2, 3])
def test_uniform_periodic_pattern_closed_form(ndim):
    """Every face of a uniform periodic mesh is SRL with the (g +- e_d) mod E neighbour."""
    level = 2
    ntrees = (2, 3, 1) if ndim == 2 else (2, 1, 2)
    sp = synth.MeshSpec(ndim=ndim, N=4, ng=2, ntrees=ntrees, periodic=(1, 1, 1), max_level=level)
    m = oracle.Mesh(sp, level)
    lev, g = m.blocks()
    index = {tuple(g[b]): b for b in range(len(lev))}
    pat = m.pattern()
    assert len(pat) == 2 * ndim * len(lev)
    assert np.all(pat[:, 0] == oracle.KIND_SRL)
    E = [ntrees[d] << level for d in range(3)]
    for kind, face, dst, src, off, aux in pat:
        d, side = divmod(face, 2)
        q = list(g[dst])
        q[d] = (q[d] + (1 if side else -1)) % E[d]
        assert src == index[tuple(q)]
        assert off == 0 and aux == 0


def leaf_boxes(sp, lev, g):
    """Integer boxes [lo, hi) of every leaf in units of the finest block."""
    L = sp.max_level
    size = 1 << (L - lev.astype(np.int64))
    lo = g[:, :sp.ndim] * size[:, None]
    return lo, lo + size[:, None]


def touches(sp, alo, ahi, blo, bhi):
    """Closed boxes intersect (periodic images included) and are distinct."""
    ext = [sp.ntrees[d] << sp.max_level for d in range(sp.ndim)]
    for shift in itertools.product(*[(-1, 0, 1) if sp.periodic[d] else (0,) for d in range(sp.ndim)]):
        ok = True
        for d in range(sp.ndim):
            s = shift[d] * ext[d]
            if blo[d] + s > ahi[d] or bhi[d] + s < alo[d]:
                ok = False
                break
        if ok:
            return True
    return False


def random_meshes(ndim, seed, rounds=4):
    rng = np.random.default_rng(seed)
    if ndim == 2:
        sp = synth.MeshSpec(ndim=2, N=4, ng=2, ntrees=(3, 2, 1), periodic=(rng.integers(2), rng.integers(2), 1), max_level=4)
    else:
        sp = synth.MeshSpec(ndim=3, N=4, ng=2, ntrees=(2, 1, 2), periodic=tuple(int(x) for x in rng.integers(0, 2, 3)), max_level=3)
    m = oracle.Mesh(sp, 1)
    out = []
    for _ in range(rounds):
        flags = rng.choice(np.array([-1, 0, 1], dtype=np.int8), size=m.n, p=[0.35, 0.4, 0.25])
        nm = m.adapt(flags)
        out.append((m, flags, nm))
        m = nm
    return sp, out


@pytest.mark.parametrize("ndim,seed", [(2, s) for s in range(6)] + [(3, s) for s in range(3)])
def test_adapt_balance_coverage(ndim, seed):
    sp, seq = random_meshes(ndim, seed)
    for old, flags, new in seq:
        lev, g = new.blocks()
        lo, hi = leaf_boxes(sp, lev, g)
        # coverage: volumes add up to the brick and leaves do not overlap
        vol = np.prod(hi - lo, axis=1).sum()
        assert vol == np.prod([sp.ntrees[d] << sp.max_level for d in range(ndim)])
        for a in range(len(lev)):
            for b in range(a + 1, len(lev)):
                assert np.any(np.minimum(hi[a], hi[b]) <= np.maximum(lo[a], lo[b])), "overlap"
        # full (corner) 2:1 balance, checked pairwise by geometry
        for a in range(len(lev)):
            for b in range(a + 1, len(lev)):
                if abs(int(lev[a]) - int(lev[b])) > 1:
                    assert not touches(sp, lo[a], hi[a], lo[b], hi[b])
        assert new.balanced()
        # each new leaf is within one level of the old leaf at its position;
        # refine flags below max_level are honoured, keep flags never coarsen
        olev, og = old.blocks()
        olo, ohi = leaf_boxes(sp, olev, og)
        for b in range(len(lev)):
            c = lo[b]
            hit = [a for a in range(len(olev)) if np.all(olo[a] <= c) and np.all(c < ohi[a])]
            assert len(hit) == 1
            a = hit[0]
            assert abs(int(lev[b]) - int(olev[a])) <= 1
            if flags[a] > 0 and olev[a] < sp.max_level:
                assert lev[b] == olev[a] + 1
            if flags[a] >= 0:
                assert lev[b] >= olev[a]


@pytest.mark.parametrize("ndim,seed", [(2, s) for s in range(6)] + [(3, s) for s in range(3)])
def test_pattern_invariants(ndim, seed):
    """Classification checked against box geometry, and every receiving face
    covered exactly once; SRL and F2C/C2F entries are reciprocal."""
    sp, seq = random_meshes(ndim, seed, rounds=3)
    m = seq[-1][2]
    lev, g = m.blocks()
    lo, hi = leaf_boxes(sp, lev, g)
    pat = m.pattern()
    ext = [sp.ntrees[d] << sp.max_level for d in range(ndim)]
    per_face = {}
    for kind, face, dst, src, off, aux in pat:
        per_face.setdefault((dst, face), []).append((kind, src, off))
    assert len(per_face) == 2 * ndim * len(lev)
    srl = set()
    f2c = set()
    c2f = set()
    nbc = 0
    for (dst, face), items in per_face.items():
        d, side = divmod(face, 2)
        kinds = {k for k, _, _ in items}
        assert len(kinds) == 1
        k = kinds.pop()
        on_boundary = (lo[dst][d] == 0 and side == 0) or (hi[dst][d] == ext[d] and side == 1)
        if k == oracle.KIND_BC:
            assert on_boundary and not sp.periodic[d] and len(items) == 1
            nbc += 1
            continue
        assert not (on_boundary and not sp.periodic[d])
        if k == oracle.KIND_F2C:
            assert len(items) == 2 ** (ndim - 1)
            assert sorted(o for _, _, o in items) == list(range(2 ** (ndim - 1)))
        else:
            assert len(items) == 1
        for _, src, off in items:
            exp_lev = {oracle.KIND_SRL: 0, oracle.KIND_F2C: 1, oracle.KIND_C2F: -1}[k]
            assert lev[src] - lev[dst] == exp_lev
            # src lies across `face`: shift dst's box by its own size along d
            size = hi[dst][d] - lo[dst][d]
            probe_lo = lo[dst].copy()
            probe_lo[d] = (probe_lo[d] + (size if side else -1)) % ext[d]
            inside = all(lo[src][e] <= probe_lo[e] < hi[src][e] for e in range(ndim) if e == d)
            assert inside
            tds = [e for e in range(ndim) if e != d]
            if k == oracle.KIND_SRL:
                assert all(lo[src][e] == lo[dst][e] for e in tds)
                srl.add((dst, face, src))
            elif k == oracle.KIND_F2C:
                pos = [(lo[src][e] - lo[dst][e]) // (hi[src][e] - lo[src][e]) for e in tds]
                assert off == sum(p << i for i, p in enumerate(pos))
                f2c.add((dst, face, src, off))
            else:
                pos = [(lo[dst][e] - lo[src][e]) // (hi[dst][e] - lo[dst][e]) for e in tds]
                assert off == sum(p << i for i, p in enumerate(pos))
                c2f.add((dst, face, src, off))
    for dst, face, src in srl:
        assert (src, face ^ 1, dst) in srl
    assert {(s, f ^ 1, d, o) for d, f, s, o in f2c} == c2f
    bc = pat[pat[:, 0] == oracle.KIND_BC]
    assert bc[:, 5].tolist() == list(range(nbc))
    # canonical order
    keys = [tuple(r) for r in pat[:, [0, 1, 2, 4]]]
    assert keys == sorted(keys)


@pytest.mark.parametrize("ndim", [2, 3])
def test_diagonal_ghosts_closed_form_on_periodic_mesh(ndim):
    """Edge and corner ghost cells (an option; the paper fills face ghosts
    only): on a uniform periodic mesh every ghost cell -- face, edge and
    corner -- holds the field of its wrapped global cell; without the option
    the edge and corner cells are left as they were."""
    nt = (3, 2, 2)[:ndim] + (1,) * (3 - ndim)
    for diag in (1, 0):
        sp = synth.MeshSpec(ndim=ndim, N=8, ng=2, ntrees=nt, diagonal_ghosts=diag)
        m = oracle.Mesh(sp, 0)
        lev, g = m.blocks()
        S, N, ng = sp.side, sp.N, sp.ng
        loc = np.arange(S) - ng
        coords = []
        for d in range(ndim):
            c = (g[:, d, None] * N + loc[None, :]) % (nt[d] * N)
            shape = [len(lev)] + [1] * ndim
            shape[ndim - d] = S
            coords.append(c.reshape(shape))
        field = sum((7.0 ** d) * coords[d] for d in range(ndim)) + 0.25
        field = np.broadcast_to(field, [len(lev)] + [S] * ndim)
        u = np.stack([(v + 1.0) * field for v in range(sp.nvar)], axis=1).reshape(len(lev), sp.nvar, -1).copy()
        u = synth.mask_interior(sp, u)
        m.fill_ghosts(u)
        U = u.reshape((len(lev), sp.nvar) + (S,) * ndim)
        F = np.stack([(v + 1.0) * field for v in range(sp.nvar)], axis=1)
        idx = np.indices((S,) * ndim) - ng
        nout = sum(((idx[d] < 0) | (idx[d] >= N)).astype(int) for d in range(ndim))
        diagonal = nout >= 2
        np.testing.assert_array_equal(U[:, :, ~diagonal], F[:, :, ~diagonal])
        if diag:
            np.testing.assert_array_equal(U[:, :, diagonal], F[:, :, diagonal])
        else:
            assert not U[:, :, diagonal].any()


@pytest.mark.parametrize("ndim,seed", [(2, 1), (2, 4), (3, 2)])
def test_diagonal_pattern_entries_geometry(ndim, seed):
    """Every diagonal entry names a same-level leaf displaced by its
    direction code (dx+1) + 3(dy+1) + 9(dz+1), with periodic wrap, and every
    such same-level neighbour has an entry."""
    import dataclasses
    sp, seq = random_meshes(ndim, seed, rounds=3)
    spd = dataclasses.replace(sp, diagonal_ghosts=1)
    m = oracle.Mesh(spd, 1)
    for _, flags, _ in seq:
        m = m.adapt(flags)
        lev, g = m.blocks()
        pat = m.pattern()
        where = {(int(a), *map(int, b)): i for i, (a, b) in enumerate(zip(lev, g))}
        expect = set()
        for b in range(m.n):
            for dz in ((-1, 0, 1) if ndim == 3 else (0,)):
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        dirs = (dx, dy, dz)
                        if sum(x != 0 for x in dirs) < 2:
                            continue
                        q, ok = [], True
                        for d in range(ndim):
                            E = spd.ntrees[d] << int(lev[b])
                            x = int(g[b][d]) + dirs[d]
                            if x < 0 or x >= E:
                                if not spd.periodic[d]:
                                    ok = False
                                    break
                                x %= E
                            q.append(x)
                        if not ok:
                            continue
                        s = where.get((int(lev[b]), *(q + [0] * (3 - ndim))))
                        if s is not None:
                            expect.add(((dx + 1) + 3 * (dy + 1) + 9 * (dz + 1), b, s))
        got = {(int(e[1]), int(e[2]), int(e[3])) for e in pat[pat[:, 0] == 4]}
        assert got == expect


@pytest.mark.parametrize("ndim,seed", [(2, 1), (2, 4), (3, 2)])
def test_diagonal_pattern_entries_across_levels(ndim, seed):
    """Edge and corner regions next to other levels: a coarser leaf holding
    the same-size box q gives one prolongation entry (kind 6) whose offset
    holds the parity of q per dimension; a refined q gives one restriction
    entry (kind 5) per child touching the block, offset = the child's
    position along a 3D edge."""
    import dataclasses
    sp, seq = random_meshes(ndim, seed, rounds=3)
    spd = dataclasses.replace(sp, diagonal_ghosts=1)
    m = oracle.Mesh(spd, 1)
    seen = {5: 0, 6: 0}
    for _, flags, _ in seq:
        m = m.adapt(flags)
        lev, g = m.blocks()
        pat = m.pattern()
        where = {(int(a), *map(int, b)): i for i, (a, b) in enumerate(zip(lev, g))}
        exp5, exp6 = set(), set()
        for b in range(m.n):
            L = int(lev[b])
            for dz in ((-1, 0, 1) if ndim == 3 else (0,)):
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        dirs = (dx, dy, dz)
                        if sum(x != 0 for x in dirs) < 2:
                            continue
                        q, ok = [], True
                        for d in range(ndim):
                            E = spd.ntrees[d] << L
                            x = int(g[b][d]) + dirs[d]
                            if x < 0 or x >= E:
                                if not spd.periodic[d]:
                                    ok = False
                                    break
                                x %= E
                            q.append(x)
                        if not ok or (L, *(q + [0] * (3 - ndim))) in where:
                            continue
                        code = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)
                        par = where.get((L - 1, *([c >> 1 for c in q] + [0] * (3 - ndim))))
                        if L > 0 and par is not None:
                            exp6.add((code, b, par, sum((q[d] & 1) << d for d in range(ndim))))
                            continue
                        ed = [d for d in range(ndim) if dirs[d] == 0]
                        for o in ((0, 1) if ed else (0,)):
                            ch = [2 * q[d] + (1 if dirs[d] < 0 else 0) if dirs[d] != 0 else 2 * q[d] + o
                                  for d in range(ndim)]
                            s = where[(L + 1, *(ch + [0] * (3 - ndim)))]
                            exp5.add((code, b, s, o))
        got5 = {tuple(int(x) for x in e[[1, 2, 3, 4]]) for e in pat[pat[:, 0] == 5]}
        got6 = {tuple(int(x) for x in e[[1, 2, 3, 4]]) for e in pat[pat[:, 0] == 6]}
        assert got5 == exp5 and got6 == exp6
        seen[5] += len(got5)
        seen[6] += len(got6)
    assert seen[5] > 0 and seen[6] > 0


@pytest.mark.parametrize("ndim", [2, 3])
def test_diagonal_ghosts_exact_for_linear_field_across_levels(ndim):
    """With edge and corner ghosts on, every edge and corner ghost cell
    inside the domain holds the linear field phi = x + 2y (+3z) at its
    centre up to rounding, whether it was copied, restricted from finer
    leaves or prolonged from a coarser one (the prolongation reads the
    coarse leaf's face ghosts, some of them boundary values): both transfers
    are exact for linear data, as in the test of Sec. 4.3."""
    sp = synth.MeshSpec(ndim=ndim, N=8, ng=2, ntrees=(2, 2, 2)[:ndim] + (1,) * (3 - ndim), periodic=(0, 0, 0),
                        max_level=3, bc_type=(3,) * 6, diagonal_ghosts=1)
    m = oracle.Mesh(sp, 0)
    for _ in range(3):
        lev, g = m.blocks()
        m = m.adapt(synth.point_flags(sp, lev, g, (0.3, 0.62, 0.45)[:ndim] + (0.0,) * (3 - ndim), 3))
    lev, g = m.blocks()
    pat = m.pattern()
    kinds = set(pat[:, 0].tolist())
    assert {4, 5, 6} <= kinds
    u = synth.linear_field(sp, lev, g)
    bce = [(f, d) for k, f, d, s, o, a in pat if k == oracle.KIND_BC]
    m.fill_ghosts(u, synth.linear_face_values(sp, lev, g, bce))
    exact = synth.linear_field(sp, lev, g, with_ghosts=True)
    X = synth.cell_centres(sp, lev, g)
    inside = np.ones_like(X[0], dtype=bool)
    for d in range(ndim):
        inside &= (X[d] > 0.0) & (X[d] < 1.0)
    S, N, ng = sp.side, sp.N, sp.ng
    idx = np.indices((S,) * ndim) - ng
    nout = sum(((idx[d] < 0) | (idx[d] >= N)).astype(int) for d in range(ndim))
    sel = (nout >= 2)[None] & inside
    U = u.reshape((m.n, sp.nvar) + (S,) * ndim)
    Ex = exact.reshape((m.n, sp.nvar) + (S,) * ndim)
    diff = np.abs(U - Ex)
    err = diff[np.broadcast_to(sel[:, None], diff.shape)].max() / np.abs(Ex).max()
    assert err < 4.5e-16 * 8, err
    assert sel.sum() > 0


@pytest.mark.parametrize("ndim", [2, 3])
def test_outside_edge_and_corner_ghosts_exact_for_linear_field(ndim):
    """Edge and corner ghost cells outside a non-periodic domain (a reading
    added here; the paper fills face ghosts only) take the boundary formula
    of the face across their lowest dimension that leaves the domain,
    applied to the cell mirrored across that face: a face ghost for an edge
    cell, an edge cell for a corner.  With Neumann values equal to the
    outward derivative of the linear field of Sec. 4.3, reflection is exact,
    so every ghost cell of every block -- face, edge and corner, inside or
    outside the domain -- holds the field, on a 4-level mesh refined toward
    a corner of the domain.  A mirror cell off by one layer, the wrong face's
    value or corners filled before edges break it."""
    coef = (1.0, 2.0, 3.0)
    bcv = tuple(tuple(((v + 1.0) * coef[f // 2] * (1.0 if f % 2 else -1.0)) if f // 2 < ndim else 0.0
                      for v in range(8)) for f in range(6))
    sp = synth.MeshSpec(ndim=ndim, N=8, ng=2, ntrees=(2, 2, 2)[:ndim] + (1,) * (3 - ndim), periodic=(0, 0, 0),
                        max_level=3, bc_type=(2,) * 6, bc_val=bcv, diagonal_ghosts=1)
    m = oracle.Mesh(sp, 0)
    for _ in range(3):
        lev, g = m.blocks()
        m = m.adapt(synth.point_flags(sp, lev, g, (0.02, 0.97, 0.03)[:ndim] + (0.0,) * (3 - ndim), 3))
    lev, g = m.blocks()
    assert int(lev.max()) == 3
    pat = m.pattern()
    diag_bc = pat[pat[:, 0] == 7]
    assert len(diag_bc) > 0
    # a boundary entry's offset names a face of its block that is a domain boundary
    bc_faces = {(int(e[2]), int(e[1])) for e in pat if e[0] == oracle.KIND_BC}
    assert all((int(e[2]), int(e[4])) in bc_faces for e in diag_bc)
    exact = synth.linear_field(sp, lev, g, with_ghosts=True)
    # every ghost cell starts far from the field, so one left unfilled fails
    S = sp.side
    idx = np.indices((S,) * ndim) - sp.ng
    nout = sum(((idx[d] < 0) | (idx[d] >= sp.N)).astype(int) for d in range(ndim))
    u = exact.copy().reshape((m.n, sp.nvar) + (S,) * ndim)
    u[:, :, nout > 0] = 1e6
    u = u.reshape(exact.shape)
    m.fill_ghosts(u)
    err = np.abs(u - exact).max() / np.abs(exact).max()
    assert err < 4.5e-16 * 16, err
    # the check covers edge and corner cells outside the domain
    X = synth.cell_centres(sp, lev, g)
    outside = np.zeros_like(X[0], dtype=bool)
    for d in range(ndim):
        outside |= (X[d] < 0.0) | (X[d] > 1.0)
    assert ((nout >= 2)[None] & outside).sum() > 0
