"""CPU-side checks of the C-ABI library: it builds, loads, exports every symbol
include/*.h declares, and rejects bad clouds before touching the GPU."""
import os
import re

import numpy as np
import pytest

from paper_2406_07441_gb300 import cloudgen as cg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lk():
    from paper_2406_07441_gb300 import build, lskum
    build.build()
    lskum.load()
    return lskum


def test_exports_every_declared_symbol(lk):
    hdr = "".join(open(os.path.join(ROOT, "include", f)).read()
                  for f in sorted(os.listdir(os.path.join(ROOT, "include"))) if f.endswith(".h"))
    names = set(re.findall(r"\b(lskum_[a-z_]+)\s*\(", hdr))
    assert len(names) >= 35
    L = lk.load()
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing


def _cloud_copy(c):
    return cg.Cloud(c.x.copy(), c.y.copy(), c.flag.copy(), c.nx.copy(), c.ny.copy(), c.nbr_off.copy(),
                    c.nbr_idx.copy(), dict(c.meta))


@pytest.mark.parametrize("defect", ["self", "range", "dup", "flag", "nan", "offsets", "normal"])
def test_bad_clouds_are_rejected_on_the_host(lk, defect):
    c = _cloud_copy(cg.naca0012_block(40, 16))
    if defect == "self":
        c.nbr_idx[c.nbr_off[5]] = 5
    elif defect == "range":
        c.nbr_idx[3] = c.n
    elif defect == "dup":
        c.nbr_idx[c.nbr_off[50] + 1] = c.nbr_idx[c.nbr_off[50]]
    elif defect == "flag":
        c.flag[9] = 7
    elif defect == "nan":
        c.x[11] = np.nan
    elif defect == "offsets":
        c.nbr_off[4] = c.nbr_off[5] + 1
    elif defect == "normal":
        c.nx[2] *= 2.0
    with pytest.raises(lk.LskumError) as ei:
        lk.Solver(c, 0.5, 1.0)
    assert ei.value.status == -1


def test_degenerate_split_stencil_is_rejected(lk):
    c = _cloud_copy(cg.cartesian_box(7, 7, seed=1))
    # an interior point whose neighbours all lie on its left: no x- sub-stencil
    p = 24
    x, y = c.x, c.y
    left = [q for q in range(c.n) if x[q] < x[p] - 1e-9 and q != p]
    left = sorted(left, key=lambda q: (x[q] - x[p]) ** 2 + (y[q] - y[p]) ** 2)[:6]
    rows = [list(c.nbr_idx[c.nbr_off[k]:c.nbr_off[k + 1]]) for k in range(c.n)]
    rows[p] = left
    off = np.zeros(c.n + 1, np.int32)
    off[1:] = np.cumsum([len(r) for r in rows])
    c.nbr_off = off
    c.nbr_idx = np.concatenate([np.array(r, np.int32) for r in rows])
    with pytest.raises(lk.LskumError) as ei:
        lk.Solver(c, 0.5, 1.0)
    assert ei.value.status == -2
    assert "point 24" in str(ei.value)


def test_bad_options_are_rejected(lk):
    c = cg.naca0012_block(40, 16)
    for kw in (dict(cfl=0.0), dict(inner_iters=-1), dict(jvp=5), dict(scheme=2), dict(scheme=1, precision=1),
               dict(farfield=2)):
        with pytest.raises(lk.LskumError) as ei:
            lk.Solver(c, 0.5, 1.0, **kw)
        assert ei.value.status == -1


def test_empty_and_isolated_clouds_are_rejected(lk):
    """No points: LSKUM_ERR_ARG; one interior point without neighbours: its
    least-squares stencil is degenerate, LSKUM_ERR_STENCIL; both before any
    device call."""
    empty = cg.Cloud(np.zeros(0), np.zeros(0), np.zeros(0, np.uint8), np.zeros(0), np.zeros(0),
                     np.zeros(1, np.int32), np.zeros(0, np.int32), {})
    with pytest.raises(lk.LskumError) as ei:
        lk.Solver(empty, 0.5, 1.0)
    assert ei.value.status == -1
    one = cg.Cloud(np.zeros(1), np.zeros(1), np.zeros(1, np.uint8), np.zeros(1), np.zeros(1),
                   np.zeros(2, np.int32), np.zeros(0, np.int32), {})
    with pytest.raises(lk.LskumError) as ei:
        lk.Solver(one, 0.5, 1.0)
    assert ei.value.status == -2


@pytest.mark.parametrize("ordering", [0, 1])
def test_host_layout_invariants_hold(lk, ordering):
    """lskum_validate builds the host layout without a device and checks its
    invariants (sweep levels independent, slot lists exactly the couplings
    of earlier / later levels, sweep orders permutations); the colour count
    equals the oracle's Alg. 5."""
    import oracle as O
    clouds = [cg.naca0012_block(40, 16), cg.naca0012_jittered(64, 32, seed=12),
              cg.cartesian_box(7, 7, seed=2, wall_bottom=True), cg.naca0012_jittered(200, 80, seed=5),
              cg.cartesian_box(9, 8, seed=3)]  # no wall: the packed sweeps' levels without framed points
    for c in clouds:
        nc, nl = lk.validate([c], [(0.5, 1.0)], ordering=ordering)
        assert nc == O.Oracle(c).ncolours
        assert nl >= nc if ordering else nl <= nc
    nc, nl = lk.validate(clouds[:2], [(0.5, 1.0), (0.7, -2.0)], ordering=ordering)
    assert nc == max(O.Oracle(c).ncolours for c in clouds[:2])


def test_validate_rejects_what_create_rejects(lk):
    c = _cloud_copy(cg.naca0012_block(40, 16))
    c.nbr_idx[3] = c.n
    with pytest.raises(lk.LskumError) as ei:
        lk.validate([c], [(0.5, 1.0)])
    assert ei.value.status == -1
    with pytest.raises(lk.LskumError) as ei:
        lk.validate([cg.naca0012_block(40, 16)], [(0.5, 1.0)], scheme=1, precision=1)
    assert ei.value.status == -1


@pytest.mark.parametrize("ordering", [0, 1])
def test_kinetic_far_field_layout(lk, ordering):
    """Under the kinetic far field every outer point is swept: in the colour
    order each colour is one level holding all its points; the invariants
    (checked by lskum_validate) hold with the outer points in the lists."""
    import oracle as O
    for c in (cg.naca0012_block(40, 16, kinetic_outer=True), cg.naca0012_jittered(64, 32, seed=12, kinetic_outer=True),
              cg.cartesian_box(7, 7, seed=2, wall_bottom=True, kinetic_outer=True)):
        nc, nl = lk.validate([c], [(1.2, 0.0)], ordering=ordering, farfield=lk.FARFIELD_KINETIC)
        assert nc == O.Oracle(c).ncolours
        assert nl == nc if ordering == 0 else nl >= nc
        nc0, nl0 = lk.validate([c], [(1.2, 0.0)], ordering=ordering)
        assert nc0 == nc and nl0 <= nl


def test_kinetic_far_field_checks_outer_normals_and_stencils(lk):
    """Outer normals are read (and must be unit) only under the kinetic far
    field, and only then must the outer points' t+, t- and n+ sub-stencils be
    well posed (LSKUM_ERR_STENCIL otherwise)."""
    c = _cloud_copy(cg.naca0012_block(40, 16, kinetic_outer=True))
    c.nx[-1] *= 2.0
    lk.validate([c], [(1.2, 0.0)])
    with pytest.raises(lk.LskumError) as ei:
        lk.validate([c], [(1.2, 0.0)], farfield=lk.FARFIELD_KINETIC)
    assert ei.value.status == -1 and "outer normal" in str(ei.value)
    # bottom-edge outer point of a box (normal (0, -1), t = (-1, 0)): keep its
    # neighbours on the left (t- side) and just one on the right, so its t+
    # sub-stencil has a single point
    b = cg.cartesian_box(7, 7, seed=2, kinetic_outer=True)
    p = 3
    assert b.flag[p] == cg.OUTER and b.nx[p] == 0.0 and b.ny[p] == -1.0
    rows = [list(b.nbr_idx[b.nbr_off[q]:b.nbr_off[q + 1]]) for q in range(b.n)]
    left = [q for q in rows[p] if b.x[q] <= b.x[p]]
    right = sorted((q for q in rows[p] if b.x[q] > b.x[p]), key=lambda q: abs(b.x[q] - b.x[p]) + abs(b.y[q] - b.y[p]))
    rows[p] = left + right[:1]
    off = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    idx = np.concatenate(rows).astype(np.int32)
    bad = cg.Cloud(b.x, b.y, b.flag, b.nx, b.ny, off, idx, {})
    lk.validate([bad], [(1.2, 0.0)])
    with pytest.raises(lk.LskumError) as ei:
        lk.validate([bad], [(1.2, 0.0)], farfield=lk.FARFIELD_KINETIC)
    assert ei.value.status == -2


def test_normals_may_be_computed_from_the_polygons(lk):
    """nx = ny = NULL: the library takes the normals from the closed wall
    (and outer) polygons in caller order; the layout is the same as with
    the generator's normals, and a polygon of fewer than 3 points or a
    mismatched pair of normal arrays is rejected."""
    c = cg.naca0012_block(40, 16, kinetic_outer=True)
    bare = cg.Cloud(c.x, c.y, c.flag, None, None, c.nbr_off, c.nbr_idx, {})
    for kw in (dict(), dict(farfield=lk.FARFIELD_KINETIC), dict(ordering=1)):
        assert lk.validate([bare], [(0.8, 1.0)], **kw) == lk.validate([c], [(0.8, 1.0)], **kw)
    half = cg.Cloud(c.x, c.y, c.flag, c.nx, None, c.nbr_off, c.nbr_idx, {})
    with pytest.raises(lk.LskumError) as ei:
        lk.validate([half], [(0.8, 1.0)])
    assert ei.value.status == -1
    b = cg.cartesian_box(7, 7, seed=2, wall_bottom=True)
    two = b.flag.copy()
    two[np.flatnonzero(two == cg.WALL)[2:]] = cg.INTERIOR  # only two wall points left
    with pytest.raises(lk.LskumError) as ei:
        lk.validate([cg.Cloud(b.x, b.y, two, None, None, b.nbr_off, b.nbr_idx, {})], [(0.5, 0.0)])
    assert ei.value.status == -1 and "polygon" in str(ei.value)


def _serial_depth(c, kinetic=False):
    """Dependency levels of the serial order (Alg. 2) computed here: wall,
    interior, outer points in index order; a point's level is one more than
    the highest level among its earlier neighbours (either direction)."""
    swept = (c.flag != cg.OUTER) | kinetic
    group = np.where(c.flag == cg.WALL, 0, np.where(c.flag == cg.INTERIOR, 1, 2))
    order = np.argsort(group, kind="stable")
    rank = np.empty(c.n, int)
    rank[order] = np.arange(c.n)
    nbrs = [set() for _ in range(c.n)]
    for p in range(c.n):
        for q in c.nbr_idx[c.nbr_off[p]:c.nbr_off[p + 1]]:
            nbrs[p].add(int(q))
            nbrs[int(q)].add(p)
    depth = np.zeros(c.n, int)
    for p in order:
        if swept[p]:
            earlier = [depth[q] + 1 for q in nbrs[p] if swept[q] and rank[q] < rank[p]]
            depth[p] = max(earlier, default=0)
    return depth[swept]


@pytest.mark.parametrize("kinetic", [False, True])
def test_serial_order_levels(lk, kinetic):
    """The serial order (Alg. 2) runs by levels of its dependency graph: the
    level count equals the longest dependency chain computed independently
    here, and the layout invariants hold (checked by lskum_validate)."""
    kw = dict(ordering=lk.ORDER_SERIAL)
    if kinetic:
        kw["farfield"] = lk.FARFIELD_KINETIC
    for c in (cg.cartesian_box(7, 7, seed=2, wall_bottom=True, kinetic_outer=True),
              cg.naca0012_block(40, 16, kinetic_outer=True), cg.naca0012_jittered(48, 20, seed=11, kinetic_outer=True)):
        nc, nl = lk.validate([c], [(0.63, 2.0)], **kw)
        assert nl == _serial_depth(c, kinetic).max() + 1
