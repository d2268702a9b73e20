"""The velocity-pressure system and its Schur-complement preconditioner (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 4.1 eliminates buoyancy from the lowest-order (RT0 x DG0) discretisation
and obtains (Eq. PressureVelocitySystem)

    A (U, P) = ( M2~ U - dt/2 D^T P ,  dt/2 c^2 D U + M3 P ),
    M2~ = M2^h (+) (1 + w_N^2) M2^z,

with the full (not lumped) velocity mass matrix.  Sec. 4.2 (Eq.
SchurComplement) preconditions it with the block factorisation

    P^-1 = [1, dt/2 M2inv D^T; 0, 1] diag(M2inv, H^^-1) [1, 0; -dt/2 c^2 D M2inv, 1]

where M2inv = 1 / diag(M2~) (Eq. LumpedMass) and H^^-1 is one V-cycle on the
lumped Helmholtz operator H^ (Eq. Preconditioner), which is exactly
M3 + w_c^2 D M2inv D^T.  The outer method is GMRES(30) (Sec. 5).

Unknowns and bases (the readings of helmholtz.py):
* horizontal faces f = edge * nz + layer, unit-flux RT0 functions; on the
  prism K over T (layer l) the function of edge k of T with outward flux +1
  is (x - v_k) / (2 |T| dz) horizontally (v_k the vertex opposite edge k),
  so  int_K w_k . w_k' = S_T[k, k'] / dz  with the scale-invariant
  S_T[k, k'] = int_T (x - v_k).(x - v_k') dA / (4 |T|^2);  the global
  function of face f is D[K, f] times the local one on each of its two cells;
* vertical faces f = col * (nz - 1) + l (between layers l and l + 1), P1 in z
  with unit flux through the face: z^ phi_f(z) / A_K on cell K, so the cell
  K (area A_K) adds dz / (3 A_K) to each of its two faces' diagonal and
  dz / (6 A_K) between them;
* pressure: DG0 per cell, M3 = diag(|K|); D entries +-1 (helmholtz.py).
"""
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from oracle import helmholtz, multigrid


def rt0_local_mass(mesh):
    """S[F, k, k'] = int_T (x - v_k).(x - v_k') dA / (4 |T|^2) on the flat
    unit-sphere triangle T = face F (scale invariant).  With barycentric
    coordinates x - v_k = sum_m lam_m (v_m - v_k) and
    int_T lam_m lam_n dA = |T| (1 + delta_mn) / 12."""
    V = mesh.verts[mesh.faces]                     # (nf, 3, 3): vertex m of face F
    area = mesh.area1
    S = np.empty((mesh.ncols, 3, 3))
    w = (np.ones((3, 3)) + np.eye(3)) / 12.0      # int lam_m lam_n / |T|
    for k in range(3):
        dk = V - V[:, k:k + 1, :]                  # v_m - v_k
        for kk in range(3):
            dkk = V - V[:, kk:kk + 1, :]
            g = np.einsum("fmi,fni->fmn", dk, dkk)     # (v_m - v_k).(v_n - v_k')
            S[:, k, kk] = np.einsum("fmn,mn->f", g, w) * area / (4.0 * area ** 2)
    return S


@dataclass
class MixedOperator:
    ncols: int
    nlayers: int
    nhf: int                  # horizontal faces
    nvf: int                  # vertical faces
    Mh: sp.csr_matrix         # M2^h
    Mz: sp.csr_matrix         # M2^z
    D: sp.csr_matrix          # cells x (horizontal + vertical faces)
    M3: np.ndarray
    a: float                  # dt / 2
    c2: float                 # c^2
    wn2: float                # w_N^2
    A: sp.csr_matrix          # the whole system matrix
    m2diag: np.ndarray        # diag(M2~)

    @property
    def nu(self):
        return self.nhf + self.nvf

    @property
    def n(self):
        return self.nu + self.M3.size


def assemble_mixed(mesh, prm):
    """A of Eq. PressureVelocitySystem on one mesh (no orography, theta = 1)."""
    op = helmholtz.assemble(mesh, prm)
    nc, nz = mesh.ncols, prm.nlayers
    ncells = nc * nz
    edges = helmholtz.horizontal_faces(mesh)
    ne = edges.shape[0]
    nhf, nvf = ne * nz, nc * (nz - 1)
    dz = prm.dz

    # edge of (column, local edge k) and the sign of D_h there
    edge_of = np.empty((nc, 3), dtype=np.int64)
    sign_of = np.empty((nc, 3))
    t, k, tn, kn = edges.T
    edge_of[t, k] = np.arange(ne)
    sign_of[t, k] = 1.0
    edge_of[tn, kn] = np.arange(ne)
    sign_of[tn, kn] = -1.0

    S = rt0_local_mass(mesh)
    rows, cols, vals = [], [], []
    for i in range(3):
        for j in range(3):
            for lay in range(nz):
                rows.append(edge_of[:, i] * nz + lay)
                cols.append(edge_of[:, j] * nz + lay)
                vals.append(sign_of[:, i] * sign_of[:, j] * S[:, i, j] / dz)
    Mh = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(nhf, nhf))

    area = mesh.area1[:, None] * prm.rho()[None, :] ** 2   # A_K
    rows, cols, vals = [], [], []
    for c in range(nc):
        for lay in range(nz):
            faces = []
            if lay > 0:
                faces.append(c * (nz - 1) + lay - 1)       # bottom face of the cell
            if lay < nz - 1:
                faces.append(c * (nz - 1) + lay)           # top face
            for f in faces:
                for g in faces:
                    rows.append(f)
                    cols.append(g)
                    vals.append(dz / (3.0 * area[c, lay]) if f == g else dz / (6.0 * area[c, lay]))
    Mz = sp.csr_matrix((vals, (rows, cols)), shape=(nvf, nvf))

    D = sp.hstack([op.Dh, op.Dz]).tocsr()
    wn2 = prm.omega_N ** 2
    M2t = sp.block_diag([Mh, (1.0 + wn2) * Mz]).tocsr()
    a = 0.5 * prm.dt
    c2 = prm.c ** 2
    A = sp.bmat([[M2t, -a * D.T], [a * c2 * D, sp.diags(op.M3)]]).tocsr()
    return MixedOperator(nc, nz, nhf, nvf, Mh, Mz, D, op.M3, a, c2, wn2, A, M2t.diagonal())


def apply_mixed(mop, x):
    return mop.A @ x


def assembled_rhs(mop, r):
    """The right-hand side (M2~ R_U, M3 R_P) of Eq. PressureVelocitySystem for
    field values r = (R_U, R_P) (faces, then cells)."""
    ru, rp = r[:mop.nu], r[mop.nu:]
    return np.concatenate([mop.A[:mop.nu, :mop.nu] @ ru, mop.M3 * rp])


def schur_precondition(mop, ops, r):
    """z = P^-1 r (Eq. SchurComplement with Eq. LumpedMass), H^^-1 = one
    V-cycle on the Helmholtz hierarchy `ops` (level 0 = this mesh)."""
    ru, rp = r[:mop.nu], r[mop.nu:]
    tu = ru / mop.m2diag                                   # M2inv r_U
    rp2 = rp - mop.a * mop.c2 * (mop.D @ tu)               # lower factor
    zp = multigrid.vcycle(ops, rp2)                        # H^^-1
    zu = tu + mop.a * (mop.D.T @ zp) / mop.m2diag          # upper factor
    return np.concatenate([zu, zp])
