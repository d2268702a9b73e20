"""Pins of the oracle's icosahedral mesh hierarchy (Sec. 3.1, Table "Grid setup")."""
import os

import numpy as np
import pytest

from oracle import helmholtz, mesh

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "grid_setup.txt")


def _edges(faces):
    e = set()
    for a, b, c in faces:
        for u, v in ((a, b), (b, c), (c, a)):
            e.add((min(u, v), max(u, v)))
    return e


@pytest.mark.parametrize("r", [0, 1, 2, 3])
def test_counts_and_euler(r):
    m = mesh.hierarchy(r, 1)[0]
    F = m.faces.shape[0]
    E = len(_edges(m.faces))
    V = len(np.unique(m.faces))
    assert F == 20 * 4 ** r
    assert E == 30 * 4 ** r
    assert V == 10 * 4 ** r + 2
    assert V - E + F == 2


@pytest.mark.parametrize("r", [0, 2, 3])
def test_vertices_on_unit_sphere_and_orientation(r):
    m = mesh.hierarchy(r, 1)[0]
    assert np.allclose(np.linalg.norm(m.verts, axis=1), 1.0, atol=1e-15)
    p0, p1, p2 = (m.verts[m.faces[:, k]] for k in range(3))
    outward = np.sum(np.cross(p1 - p0, p2 - p0) * (p0 + p1 + p2), axis=1)
    assert np.all(outward > 0)


@pytest.mark.parametrize("r", [0, 1, 3])
def test_neighbours_symmetric_and_share_the_opposite_edge(r):
    m = mesh.hierarchy(r, 1)[0]
    for f in range(m.ncols):
        nb = m.nbr[f]
        assert len(set(nb.tolist())) == 3 and f not in nb
        for k in range(3):
            g = nb[k]
            assert f in m.nbr[g]
            shared = set(m.faces[f].tolist()) & set(m.faces[g].tolist())
            edge = {m.faces[f][(k + 1) % 3], m.faces[f][(k + 2) % 3]}
            assert shared == edge


def test_children_are_nested_in_parent():
    fine, coarse = mesh.hierarchy(3, 2)
    for F in range(coarse.ncols):
        parent = coarse.faces[F]
        kids = fine.faces[4 * F: 4 * F + 4]
        # corner child j holds parent vertex j (same coordinates)
        for j in range(3):
            assert np.any(np.all(np.isclose(fine.verts[kids[j]], coarse.verts[parent[j]]), axis=1))
        # the centre child's vertices are the three edge midpoints
        mids = set()
        for j in range(3):
            a, b = coarse.verts[parent[j]], coarse.verts[parent[(j + 1) % 3]]
            m = (a + b) / np.linalg.norm(a + b)
            assert np.any(np.all(np.isclose(fine.verts[kids[3]], m), axis=1))
        # children tile the parent: their flat areas sum to ~ the parent's
        # (exactly in the plane; the midpoints are lifted to the sphere)
        assert fine.area1[4 * F: 4 * F + 4].sum() == pytest.approx(coarse.area1[F], rel=0.2)


def test_area_increases_towards_sphere():
    areas = [mesh.hierarchy(r, 1)[0].area1.sum() for r in range(6)]
    assert all(a < 4 * np.pi for a in areas)
    assert all(b > a for a, b in zip(areas, areas[1:]))
    # a chord triangle with edge h loses O(h^2) area to the sphere
    deficits = [4 * np.pi - a for a in areas]
    for d0, d1 in zip(deficits[2:], deficits[3:]):
        assert d1 / d0 == pytest.approx(0.25, abs=0.02)


def test_grid_setup_table():
    """Table "Grid setup": 81,920 LO columns with dx ~ 90 km, 5,120 NLO
    columns with dx ~ 360 km, 64 layers, 3.5 LO unknowns per cell, 18.4 mio."""
    rows = [ln.split() for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")]
    lo = next(r for r in rows if r[0] == "LO")
    nlo = next(r for r in rows if r[0] == "NLO")
    cells_lo, dx_lo, nz, per_cell, total = int(lo[1]), float(lo[2]), int(lo[3]), float(lo[4]), float(lo[5])
    # LO grid: refinement 6
    m6 = mesh.hierarchy(6, 1)[0]
    assert m6.ncols == cells_lo
    E = helmholtz.horizontal_faces(m6).shape[0]
    # pressure (DG0): 1 per cell; horizontal RT0 flux: E per layer; vertical
    # flux: one face per cell (interior faces plus one boundary layer)
    unknowns = m6.ncols * nz + E * nz + m6.ncols * nz
    assert unknowns / (m6.ncols * nz) == per_cell
    assert round(unknowns / 1e6, 1) == total
    assert helmholtz.Params(refinement=6, nlayers=nz).dx == pytest.approx(dx_lo * 1e3)
    # NLO grid: refinement 4
    assert 20 * 4 ** 4 == int(nlo[1])
    assert mesh.hierarchy(4, 1)[0].ncols == int(nlo[1])
    assert helmholtz.Params(refinement=4, nlayers=nz).dx == pytest.approx(float(nlo[2]) * 1e3)
