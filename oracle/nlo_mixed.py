"""The next-to-lowest-order velocity-pressure system and its Schur-complement
preconditioner (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Eq. (PressureVelocitySystem) with the NLO spaces of Table "FiniteElements"
(the readings of oracle/nlo.py):

    A (U, P) = ( M2~ U - dt/2 D^T P ,  dt/2 c^2 D U + M3 P ),
    M2~ = M2^h (+) (1 + w_N^2) M2^z,

with the full (consistent) velocity masses: M2^h of BDFM1(T) x DG1(z) and
M2^z of DG1(T) x P2(z), D = [D_h, D_z] and M3 the DG1 x DG1 pressure mass,
all from nlo.assemble_nlo's unknowns and basis functions.  Eq.
(SchurComplement) preconditions it with M2inv = 1 / diag(M2~) (Eq.
LumpedMass) and one NLO V-cycle (nlo.vcycle) for H^^-1; M3 + w_c^2 D M2inv
D^T is exactly the NLO operator H^.  Unknown order: horizontal velocity
(nlo.horizontal_dofs), vertical velocity (column, vertex i, node 1 ..
2 nz - 1), pressure (nlo.pdof).
"""
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from oracle import nlo


@dataclass
class NLOMixed:
    nhf: int
    nvf: int
    npr: int
    Mh: sp.csr_matrix
    Mz: sp.csr_matrix
    D: sp.csr_matrix
    M3: sp.csr_matrix
    a: float
    c2: float
    wn2: float
    A: sp.csr_matrix
    m2diag: np.ndarray

    @property
    def nu(self):
        return self.nhf + self.nvf

    @property
    def n(self):
        return self.nu + self.npr


def velocity_masses(mesh, prm):
    """(M2^h, M2^z): the consistent masses of the horizontal and vertical
    velocity functions of nlo.assemble_nlo (horizontal v_a(x) psi_b(z) / dz,
    vertical z^ lam_i(x) zeta_n(z) / (2 |T_l|)), prism over T scaled to the
    mid-layer radius."""
    nc, nz, dz = mesh.ncols, prm.nlayers, prm.dz
    rho = prm.rho()
    owner, nhe, nhf = nlo.horizontal_dofs(mesh, nz)
    local = [dict() for _ in range(nc)]              # column -> local unknown a -> (base, sign)
    for (c, a, base, sgn) in owner:
        local[c][a] = (base, sgn)
    rows, cols, vals = [], [], []
    lay = np.arange(nz)
    for c in range(nc):
        T = nlo.triangle_bdfm(mesh.verts[mesh.faces[c]])
        for a in range(9):
            ba, sa = local[c][a]
            for a2 in range(9):
                b2, s2 = local[c][a2]
                for b in range(2):
                    for bb in range(2):
                        rows.append(ba + 2 * lay + b)
                        cols.append(b2 + 2 * lay + bb)
                        vals.append(np.full(nz, sa * s2 * T.mass[a, a2] * nlo.MZ1[b, bb] / dz))
    Mh = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(nhf, nhf))

    PM = np.array([[2.0, 1.0, 1.0], [1.0, 2.0, 1.0], [1.0, 1.0, 2.0]]) / 12.0   # int_T lam lam' / |T|
    nzn = 2 * nz - 1
    nvf = nc * 3 * nzn
    rows, cols, vals = [], [], []
    for c in range(nc):
        for layer in range(nz):
            At = mesh.area1[c] * rho[layer] ** 2
            for kz in range(3):
                node = 2 * layer + kz
                if node == 0 or node == 2 * nz:
                    continue
                for kz2 in range(3):
                    node2 = 2 * layer + kz2
                    if node2 == 0 or node2 == 2 * nz:
                        continue
                    for i in range(3):
                        for i2 in range(3):
                            rows.append((c * 3 + i) * nzn + node - 1)
                            cols.append((c * 3 + i2) * nzn + node2 - 1)
                            # int lam_i lam_i' / (4 |T|^2) dA * int zeta zeta' dz
                            vals.append(PM[i, i2] / (4.0 * At) * dz * nlo.MP2[kz, kz2])
    Mz = sp.csr_matrix((vals, (rows, cols)), shape=(nvf, nvf))
    return Mh, Mz


def assemble_nlo_mixed(mesh, prm, nop):
    """A of Eq. (PressureVelocitySystem) at NLO (theta = 1); nop is
    nlo.assemble_nlo(mesh, prm)."""
    Mh, Mz = velocity_masses(mesh, prm)
    D = sp.hstack([nop.Dh, nop.Dz]).tocsr()
    wn2 = prm.omega_N ** 2
    M2t = sp.block_diag([Mh, (1.0 + wn2) * Mz]).tocsr()
    a = 0.5 * prm.dt
    c2 = prm.c ** 2
    A = sp.bmat([[M2t, -a * D.T], [a * c2 * D, nop.M3]]).tocsr()
    return NLOMixed(Mh.shape[0], Mz.shape[0], nop.n, Mh, Mz, D, nop.M3, a, c2, wn2, A, M2t.diagonal())


def apply_mixed(mop, x):
    return mop.A @ x


def assembled_rhs(mop, r):
    """(M2~ R_U, M3 R_P) for field values r = (R_U, R_P)."""
    ru, rp = r[:mop.nu], r[mop.nu:]
    return np.concatenate([mop.A[:mop.nu, :mop.nu] @ ru, mop.M3 @ rp])


def schur_precondition(mop, nop, lo_ops, r):
    """z = P^-1 r (Eq. SchurComplement with Eq. LumpedMass); H^^-1 is one NLO
    V-cycle (NLO level, p-coarsening, the lowest-order hierarchy lo_ops)."""
    ru, rp = r[:mop.nu], r[mop.nu:]
    tu = ru / mop.m2diag
    rp2 = rp - mop.a * mop.c2 * (mop.D @ tu)
    zp = nlo.vcycle(nop, lo_ops, rp2)
    zu = tu + mop.a * (mop.D.T @ zp) / mop.m2diag
    return np.concatenate([zu, zp])
