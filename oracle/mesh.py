"""Icosahedral sphere meshes and their nested hierarchy (oracle).

Sec. 3.1 ("Grid hierarchies"): the multigrid needs a hierarchy of regularly
refined meshes together with the fine-to-coarse cell relation.  The paper's
horizontal grid is Firedrake's icosahedral sphere mesh (listing of the
two-grid demo, Sec. 3) and Sec. 4.1 extrudes it radially into a thin shell.

Conventions of this oracle (the CUDA library follows the same written
conventions with its own code, and the tests match cells by centroid, so
nothing here has to agree bit for bit):

* base icosahedron: the 12 points (+-1, +-phi, 0), (0, +-1, +-phi),
  (+-phi, 0, +-1) in the order of ``_ICO_POINTS``, normalised to the unit
  sphere; its 20 faces are the vertex triples at mutual distance 2,
  sorted lexicographically, each oriented counter-clockwise seen from
  outside (first vertex = smallest index);
* refinement: a face (a, b, c) with edge midpoints m_ab, m_bc, m_ca
  (projected to the sphere) has children 4F+0 = (a, m_ab, m_ca),
  4F+1 = (m_ab, b, m_bc), 4F+2 = (m_ca, m_bc, c), 4F+3 = (m_bc, m_ca, m_ab),
  so the parent of fine cell f is f // 4;
* neighbour k of a face is the face across the edge opposite vertex k.

Geometry is that of the flat (chord) triangles on the unit sphere; the
shell's radius enters through the helmholtz module.
"""
from dataclasses import dataclass

import numpy as np

_PHI = (1.0 + np.sqrt(5.0)) / 2.0
_ICO_POINTS = [
    (-1.0, _PHI, 0.0), (1.0, _PHI, 0.0), (-1.0, -_PHI, 0.0), (1.0, -_PHI, 0.0),
    (0.0, -1.0, _PHI), (0.0, 1.0, _PHI), (0.0, -1.0, -_PHI), (0.0, 1.0, -_PHI),
    (_PHI, 0.0, -1.0), (_PHI, 0.0, 1.0), (-_PHI, 0.0, -1.0), (-_PHI, 0.0, 1.0),
]


def icosahedron():
    """The 12 vertices (unit sphere) and 20 counter-clockwise faces."""
    pts = np.array(_ICO_POINTS, dtype=np.float64)
    faces = []
    for i in range(12):
        for j in range(i + 1, 12):
            for k in range(j + 1, 12):
                dij = np.linalg.norm(pts[i] - pts[j])
                djk = np.linalg.norm(pts[j] - pts[k])
                dik = np.linalg.norm(pts[i] - pts[k])
                if abs(dij - 2.0) < 1e-9 and abs(djk - 2.0) < 1e-9 and abs(dik - 2.0) < 1e-9:
                    n = np.cross(pts[j] - pts[i], pts[k] - pts[i])
                    if np.dot(n, pts[i] + pts[j] + pts[k]) > 0:
                        faces.append((i, j, k))
                    else:
                        faces.append((i, k, j))
    verts = pts / np.linalg.norm(pts, axis=1, keepdims=True)
    return verts, np.array(faces, dtype=np.int64)


def refine(verts, faces):
    """Split every triangle into four at its edge midpoints (Sec. 3.1).

    New vertices are the chord midpoints projected radially onto the unit
    sphere.  Returns (verts, faces) with the children of face F at 4F..4F+3.
    """
    midpoint_of = {}
    new_verts = [v for v in verts]

    def midpoint(i, j):
        key = (min(i, j), max(i, j))
        if key not in midpoint_of:
            m = verts[i] + verts[j]
            m = m / np.sqrt(np.dot(m, m))
            midpoint_of[key] = len(new_verts)
            new_verts.append(m)
        return midpoint_of[key]

    children = []
    for a, b, c in faces:
        mab, mbc, mca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
        children.append((a, mab, mca))
        children.append((mab, b, mbc))
        children.append((mca, mbc, c))
        children.append((mbc, mca, mab))
    return np.array(new_verts), np.array(children, dtype=np.int64)


def neighbours(faces):
    """nbr[F, k] = the face sharing the edge opposite vertex k of face F."""
    owner = {}
    for f, tri in enumerate(faces):
        for k in range(3):
            a, b = tri[(k + 1) % 3], tri[(k + 2) % 3]
            owner.setdefault((min(a, b), max(a, b)), []).append(f)
    nbr = np.empty(faces.shape, dtype=np.int64)
    for f, tri in enumerate(faces):
        for k in range(3):
            a, b = tri[(k + 1) % 3], tri[(k + 2) % 3]
            pair = owner[(min(a, b), max(a, b))]
            assert len(pair) == 2, "mesh is not a closed manifold"
            nbr[f, k] = pair[0] if pair[1] == f else pair[1]
    return nbr


def flat_area(verts, faces):
    """Area of each flat (chord) triangle on the unit sphere."""
    p0, p1, p2 = verts[faces[:, 0]], verts[faces[:, 1]], verts[faces[:, 2]]
    return 0.5 * np.linalg.norm(np.cross(p1 - p0, p2 - p0), axis=1)


def shape_factor(verts, faces):
    """sigma[F, k] = integral over T of |w|^2 for the unit-flux RT0 function of
    the edge opposite vertex k (Sec. 4.1, lowest-order RT0 horizontal space).

    With p the vertex opposite the edge and a, b the edge vectors from p, the
    unit-flux RT0 function is w = (x - p) / (2|T|), and integrating the
    quadratic |x - p|^2 over T gives |T| (|a|^2 + |b|^2 + a.b) / 6, hence
    sigma = (|a|^2 + |b|^2 + a.b) / (24 |T|).  Scale invariant.
    """
    area = flat_area(verts, faces)
    sigma = np.empty(faces.shape, dtype=np.float64)
    for k in range(3):
        p = verts[faces[:, k]]
        a = verts[faces[:, (k + 1) % 3]] - p
        b = verts[faces[:, (k + 2) % 3]] - p
        sigma[:, k] = (np.sum(a * a, 1) + np.sum(b * b, 1) + np.sum(a * b, 1)) / (24.0 * area)
    return sigma


@dataclass
class Mesh2D:
    refinement: int
    verts: np.ndarray     # (nv, 3) unit sphere
    faces: np.ndarray     # (nf, 3) vertex ids, counter-clockwise
    nbr: np.ndarray       # (nf, 3) face across the edge opposite vertex k
    area1: np.ndarray     # (nf,) flat-triangle area on the unit sphere
    sigma: np.ndarray     # (nf, 3) RT0 shape factor of edge k
    centroid: np.ndarray  # (nf, 3) flat centroid on the unit sphere

    @property
    def ncols(self):
        return self.faces.shape[0]


def make_mesh(verts, faces, refinement):
    return Mesh2D(
        refinement=refinement,
        verts=verts,
        faces=faces,
        nbr=neighbours(faces),
        area1=flat_area(verts, faces),
        sigma=shape_factor(verts, faces),
        centroid=(verts[faces[:, 0]] + verts[faces[:, 1]] + verts[faces[:, 2]]) / 3.0,
    )


def hierarchy(refinement, nlevels):
    """Meshes of refinements refinement, refinement-1, ... (finest first).

    Level 0 is the finest; the parent of column c on level l is column c // 4
    on level l + 1 (Sec. 3.1: nested, hierarchically refined meshes).
    """
    if not 1 <= nlevels <= refinement + 1:
        raise ValueError("need 1 <= nlevels <= refinement + 1")
    verts, faces = icosahedron()
    per_refinement = [(verts, faces)]
    for _ in range(refinement):
        verts, faces = refine(verts, faces)
        per_refinement.append((verts, faces))
    levels = []
    for lev in range(nlevels):
        r = refinement - lev
        v, f = per_refinement[r]
        levels.append(make_mesh(v, f, r))
    return levels
