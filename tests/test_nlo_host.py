"""CPU parity of the library's host assembly of the next-to-lowest-order
operator (hmg_nlo_host_blocks: reference BDFM1 element mapped by the
contravariant Piola map, quadrature) against the oracle (oracle/nlo.py:
the element built on each physical triangle, exact monomial integrals).
No GPU: the assembly is host code.  Columns are matched by centroid and the
DG1 unknowns of a column by vertex position."""
import numpy as np
import pytest

from oracle import helmholtz, mesh, nlo


@pytest.fixture(scope="module")
def hmg():
    from paper_1605_00492_gb300 import build
    build.build()
    import paper_1605_00492_gb300 as lib
    return lib


@pytest.mark.parametrize("r,nz,cfl", [(1, 3, 8.0), (2, 4, 8.0), (2, 2, 32.0)])
def test_nlo_host_blocks_match_oracle(hmg, r, nz, cfl):
    B = hmg.nlo_host_blocks(r, nz, nu_cfl=cfl)
    m = mesh.hierarchy(r, 1)[0]
    prm = helmholtz.Params(refinement=r, nlayers=nz, nu_cfl=cfl)
    H = nlo.assemble_nlo(m, prm).H.tocsr()
    cen = B["verts"].mean(axis=1)
    d = np.linalg.norm(cen[:, None, :] - m.centroid[None, :, :], axis=2)
    perm = d.argmin(axis=1)
    assert np.all(d.min(axis=1) < 1e-12) and len(set(perm)) == m.ncols
    vp = np.empty((m.ncols, 3), dtype=np.int64)
    for c in range(m.ncols):
        Vo = m.verts[m.faces[perm[c]]]
        for j in range(3):
            dv = np.linalg.norm(Vo - B["verts"][c, j], axis=1)
            assert dv.min() < 1e-12
            vp[c, j] = dv.argmin()
    # the library's neighbour table is the oracle's, permuted
    for c in range(m.ncols):
        assert sorted(perm[B["nbr"][c]]) == sorted(m.nbr[perm[c]])

    # the library's blocks as one sparse matrix in the oracle's numbering
    nc = m.ncols
    u = np.arange(6)
    dof = lambda c, layer: (((perm[c][..., None] * nz + layer[..., None]) * 3 + vp[c][..., u // 2]) * 2 + u % 2)
    cc, ll = np.meshgrid(np.arange(nc), np.arange(nz), indexing="ij")
    rows = dof(cc, ll)                                          # (nc, nz, 6)
    R, C, V = [], [], []

    def add(blocks, rws, cols):
        R.append(np.broadcast_to(rws[..., :, None], blocks.shape).reshape(-1))
        C.append(np.broadcast_to(cols[..., None, :], blocks.shape).reshape(-1))
        V.append(blocks.reshape(-1))
    add(B["diag"], rows, rows)
    add(B["sub"][:, 1:], rows[:, 1:], rows[:, :-1])
    add(B["sub"][:, 1:].transpose(0, 1, 3, 2), rows[:, :-1], rows[:, 1:])   # H^ is symmetric
    assert not B["sub"][:, 0].any()
    for k in range(3):
        nb = B["nbr"][:, k]
        add(np.broadcast_to(B["nbr_blocks"][:, None, k], (nc, nz, 6, 6)), rows, dof(nb[cc], ll))
    import scipy.sparse as sp
    G = sp.csr_matrix((np.concatenate(V), (np.concatenate(R), np.concatenate(C))), shape=H.shape)
    # every block entry matches to 1e-13 of its block's largest entry (blocks
    # span several orders of magnitude, so compare each row of blocks on its own scale)
    D = (G - H).tocsr()
    scale = np.abs(H).max(axis=1).toarray().ravel()
    assert np.all(np.abs(D).max(axis=1).toarray().ravel() <= 1e-13 * scale)
    assert G.nnz == H.nnz


def test_nlo_host_blocks_argument_errors(hmg):
    with pytest.raises(hmg.HMGError):
        hmg.nlo_host_blocks(1, 0)
    with pytest.raises(hmg.HMGError):
        hmg.nlo_host_blocks(1, 3, omega=2.5)


@pytest.mark.parametrize("r,nz", [(1, 3), (2, 2)])
def test_nlo_mixed_host_csr_matches_oracle(hmg, r, nz):
    """The library's host CSR of the NLO velocity-pressure matrix (element
    matrices from the Piola-mapped reference element) against the oracle's
    assembled A, after matching the unknowns and their signs."""
    from oracle import nlo_mixed
    from tests.helpers import nlo_mixed_permutation
    A, edges = hmg.nlo_mixed_host_csr(r, nz)
    B = hmg.nlo_host_blocks(r, nz)
    m = mesh.hierarchy(r, 1)[0]
    prm = helmholtz.Params(refinement=r, nlayers=nz)
    nop = nlo.assemble_nlo(m, prm)
    mop = nlo_mixed.assemble_nlo_mixed(m, prm, nop)
    idx, sgn = nlo_mixed_permutation(B["verts"].mean(axis=1), B["verts"], edges, m, nz)
    assert A.shape == mop.A.shape and len(np.unique(idx)) == A.shape[0]
    import scipy.sparse as sp
    S = sp.diags(sgn)
    Ao = (S @ mop.A[idx][:, idx] @ S).tocsr()
    D = (A - Ao).tocsr()
    scale = np.abs(Ao).max(axis=1).toarray().ravel()
    assert np.all(np.abs(D).max(axis=1).toarray().ravel() <= 1e-12 * scale)
    assert A.nnz == Ao.nnz
