"""Test infrastructure: match the CUDA library's cells to the oracle's.

Both sides number columns by their own mesh generators; cells are matched by
the flat-triangle centroid of their column (unique to ~1e-9) and the layer.
"""
import numpy as np
from scipy.spatial import cKDTree


def column_permutation(centroids_gpu, centroids_oracle):
    """perm[g] = oracle column of GPU column g."""
    tree = cKDTree(centroids_oracle)
    dist, perm = tree.query(centroids_gpu, k=1)
    assert np.all(dist < 1e-9), f"unmatched columns (max distance {dist.max():.3e})"
    assert len(np.unique(perm)) == len(perm), "column matching is not a bijection"
    return perm


def cell_permutation(col_perm, nlayers):
    """Index array idx with v_gpu = v_oracle[idx] (COLUMN layout on both)."""
    return (np.asarray(col_perm)[:, None] * nlayers + np.arange(nlayers)[None, :]).reshape(-1)


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def nlo_unknown_maps(lib_centroids, lib_verts, mesh, nz):
    """Column permutation and vertex permutation between the library's NLO
    unknowns and the oracle's: perm[c] = oracle column of library column c,
    vp[c, j] = oracle vertex (of that face) of library vertex j."""
    perm = column_permutation(lib_centroids, mesh.centroid)
    vp = np.empty((len(perm), 3), dtype=np.int64)
    for c in range(len(perm)):
        d = np.linalg.norm(mesh.verts[mesh.faces[perm[c]]][None, :, :] - lib_verts[c][:, None, :], axis=2)
        assert d.min(axis=1).max() < 1e-12
        vp[c] = d.argmin(axis=1)
    return perm, vp


def nlo_mixed_permutation(lib_centroids, lib_verts, lib_edges, mesh, nz):
    """(idx, sign): library unknown g of the NLO velocity-pressure system is
    sign[g] times oracle unknown idx[g] (oracle/nlo_mixed.py ordering).
    Edge points are matched by position, interior (Whitney) unknowns by the
    edge and its orientation, vertical and pressure unknowns by column and
    vertex."""
    from oracle import helmholtz, nlo
    perm, vp = nlo_unknown_maps(lib_centroids, lib_verts, mesh, nz)
    nc = len(perm)
    oedges = helmholtz.horizontal_faces(mesh)
    ne = len(oedges)
    oindex = {(int(t), int(tn)): e for e, (t, k, tn, kn) in enumerate(oedges)}
    nhe = ne * 2 * nz * 2
    lay = np.arange(nz)
    idx, sign = [], []
    s13 = (1.0 / 3.0, 2.0 / 3.0)
    # horizontal edge unknowns ((E nz + l) 2 + q) 2 + b
    for E, (t, k, tn, kn) in enumerate(lib_edges):
        a, b_ = int(perm[t]), int(perm[tn])
        eo = oindex[(min(a, b_), max(a, b_))]
        to, ko = int(oedges[eo][0]), int(oedges[eo][1])
        Vl = lib_verts[t]
        Vo = mesh.verts[mesh.faces[to]]
        qmap = []
        for q in range(2):
            x = Vl[(k + 1) % 3] + s13[q] * (Vl[(k + 2) % 3] - Vl[(k + 1) % 3])
            xo = [Vo[(ko + 1) % 3] + s13[qo] * (Vo[(ko + 2) % 3] - Vo[(ko + 1) % 3]) for qo in range(2)]
            d = [np.linalg.norm(x - y) for y in xo]
            assert min(d) < 1e-12
            qmap.append(int(np.argmin(d)))
        sg = 1.0 if a == to else -1.0
        block = np.empty((nz, 2, 2), dtype=np.int64)
        for q in range(2):
            for b in range(2):
                block[:, q, b] = ((eo * 2 + qmap[q]) * nz + lay) * 2 + b
        idx.append(block.reshape(-1))
        sign.append(np.full(block.size, sg))
    # interior unknowns ((c nz + l) 3 + k) 2 + b
    for c in range(nc):
        co = int(perm[c])
        blk = np.empty((nz, 3, 2), dtype=np.int64)
        sg = np.empty((nz, 3, 2))
        for k in range(3):
            ko = int(vp[c, k])                      # the edge opposite the same vertex
            same = int(vp[c, (k + 1) % 3]) == (ko + 1) % 3
            for b in range(2):
                blk[:, k, b] = nhe + ((co * 3 + ko) * nz + lay) * 2 + b
                sg[:, k, b] = 1.0 if same else -1.0
        idx.append(blk.reshape(-1))
        sign.append(sg.reshape(-1))
    nhf = nhe + nc * 3 * nz * 2
    nzn = 2 * nz - 1
    for c in range(nc):
        for i in range(3):
            idx.append(nhf + (int(perm[c]) * 3 + int(vp[c, i])) * nzn + np.arange(nzn))
            sign.append(np.ones(nzn))
    nvf = nc * 3 * nzn
    u = np.arange(6)
    pidx = (((perm[:, None, None] * nz + lay[None, :, None]) * 3 + vp[:, None, u // 2]) * 2 + u % 2).reshape(-1)
    idx.append(nhf + nvf + pidx)
    sign.append(np.ones(pidx.size))
    assert nlo is not None
    return np.concatenate(idx), np.concatenate(sign)
