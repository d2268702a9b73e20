"""Lumped pressure-Helmholtz operator H^ of the LO (RT0 x DG0) discretisation.

Sec. 4.2, Eq. (Preconditioner):

    H^ = M3 + w_c^2 ( D_h Mh_inv D_h^T + 1/(1 + w_N^2) D_z Mz_inv D_z^T ),

with w_c = c dt / 2 (Eq. HelmholtzOperator), w_N = N dt / 2
(Eq. PressureVelocitySystem) and the lumped inverse masses of
Eq. (LumpedMass): (M_inv)_ff = 1 / M_ff.  Its column block H^_z of
Eq. (HHgeneralbanded) keeps M3, the part of D_h Mh_inv D_h^T that couples
cells of the same column (Delta_h) and the whole vertical term.

Readings of the paper used here (the paper leaves them open):

* geometry: cell K = (T, l) is the straight prism over the flat triangle T
  scaled to the mid-layer radius rho_l = R + (l + 1/2) dz, so
  |K| = A1_T rho_l^2 dz with A1_T the unit-sphere flat-triangle area;
* basis: the RT0 / P1-in-z velocity functions carry unit flux through
  their face, so D_h, D_z have entries +-1 (the product D M_inv D^T does
  not depend on that scaling); top and bottom faces carry no dof
  (u.n = 0, Eq. BoundaryCondition);
* horizontal lumped mass of a lateral face shared by prisms over T and T'
  at one layer:  Mh_ff = (sigma_T,e + sigma_T',e) / dz  (mesh.shape_factor);
* vertical lumped mass of the face between layers l and l+1 of column T:
  Mz_ff = dz / (3 A_T(rho_l) theta_l) + dz / (3 A_T(rho_l+1) theta_l+1),
  the integral of |w|^2 for w = z^ phi(z) / A over the two cells, each
  cell's contribution divided by the coefficient theta (theta = 1 unless
  the differentiable form sets it);
* dx for the Courant number: dx = 90 km * 2^(6 - r) for the finest
  refinement r (the paper prints dx ~ 90 km at 81,920 cells), with
  dt = nu_CFL dx / c shared by all levels; coarse levels are rediscretised
  on their own meshes (Sec. 3.3).
"""
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp


@dataclass
class Params:
    refinement: int                  # finest refinement r
    nlayers: int
    radius: float = 6.371e6          # m
    thickness: float = 1.0e4         # m
    c: float = 300.0                 # speed of sound, m/s  (Sec. 4.1)
    N: float = 0.01                  # buoyancy frequency, 1/s  (Sec. 4.1)
    nu_cfl: float = 8.0              # horizontal acoustic Courant number (Sec. 5)
    dx: float = None                 # m; default 90 km * 2^(6 - refinement)
    omega: float = 0.8               # over-relaxation of the smoother (Sec. 5)

    def __post_init__(self):
        if self.dx is None:
            self.dx = 90.0e3 * 2.0 ** (6 - self.refinement)

    @property
    def dz(self):
        return self.thickness / self.nlayers

    @property
    def dt(self):
        return self.nu_cfl * self.dx / self.c

    @property
    def omega_c(self):
        return 0.5 * self.c * self.dt

    @property
    def omega_N(self):
        return 0.5 * self.N * self.dt

    def rho(self):
        """Mid-layer radii R + (l + 1/2) dz."""
        return self.radius + (np.arange(self.nlayers) + 0.5) * self.dz


def cell(col, layer, nlayers):
    """Column-contiguous cell number (Sec. 4.3: all unknowns of a column are
    stored consecutively)."""
    return col * nlayers + layer


@dataclass
class Operator:
    """All matrices of one level.  Cell order: cell(col, layer)."""
    ncols: int
    nlayers: int
    M3: np.ndarray            # cell volumes |K|
    Dh: sp.csr_matrix         # cells x horizontal faces, entries +-1
    mh: np.ndarray            # lumped horizontal masses Mh_ff
    Dz: sp.csr_matrix         # cells x interior vertical faces, entries +-1
    mz: np.ndarray            # lumped vertical masses Mz_ff
    H: sp.csr_matrix          # H^
    Hz: sp.csr_matrix         # H^_z (column block-diagonal part)
    Hz_diag: np.ndarray = field(default=None)   # (ncols, nlayers)
    Hz_sub: np.ndarray = field(default=None)    # (ncols, nlayers); [:, 0] = 0

    @property
    def ncells(self):
        return self.ncols * self.nlayers


def horizontal_faces(mesh):
    """Unique edges of the 2-D mesh as rows (T, k, T', k') with T < T'."""
    nc = mesh.ncols
    t = np.repeat(np.arange(nc), 3)
    k = np.tile(np.arange(3), nc)
    tn = mesh.nbr.reshape(-1)
    keep = t < tn
    t, k, tn = t[keep], k[keep], tn[keep]
    kn = np.argmax(mesh.nbr[tn] == t[:, None], axis=1)
    assert np.all(mesh.nbr[tn, kn] == t)
    return np.stack([t, k, tn, kn], axis=1)


def assemble(mesh, prm, theta=None):
    """Build H^ and H^_z on one level (Eq. Preconditioner, Eq. HHgeneralbanded).

    theta: optional per-cell coefficient (ncells,) dividing each cell's
    contribution to the vertical lumped mass; may be complex (complex-step
    derivative checks).
    """
    nc, nz = mesh.ncols, prm.nlayers
    ncells = nc * nz
    dz = prm.dz
    rho = prm.rho()
    dtype = np.complex128 if (theta is not None and np.iscomplexobj(theta)) else np.float64
    if theta is None:
        theta = np.ones(ncells)
    theta = np.asarray(theta).reshape(nc, nz)
    layers = np.arange(nz)

    # M3: DG0 pressure mass, the cell volumes.
    area = mesh.area1[:, None] * rho[None, :] ** 2          # A_T(rho_l)
    M3 = (area * dz).reshape(-1)

    # Horizontal faces: one per (edge, layer), face number edge * nz + layer;
    # D_h = +1 on the cell over T, -1 on the cell over T'.
    edges = horizontal_faces(mesh)
    ne = edges.shape[0]
    t, k, tn, kn = edges.T
    mh = np.repeat((mesh.sigma[t, k] + mesh.sigma[tn, kn]) / dz, nz)
    f = np.arange(ne * nz)
    lay = np.tile(layers, ne)
    rows = np.concatenate([cell(np.repeat(t, nz), lay, nz), cell(np.repeat(tn, nz), lay, nz)])
    cols = np.concatenate([f, f])
    vals = np.concatenate([np.ones(ne * nz), -np.ones(ne * nz)])
    Dh = sp.csr_matrix((vals, (rows, cols)), shape=(ncells, ne * nz))

    # Vertical interior faces between layers l and l+1 of every column,
    # face number col * (nz - 1) + l; D_z = +1 below, -1 above.
    nvf = nc * (nz - 1)
    mz = (dz / (3.0 * area[:, :-1] * theta[:, :-1]) + dz / (3.0 * area[:, 1:] * theta[:, 1:])).reshape(-1)
    mz = mz.astype(dtype)
    col = np.repeat(np.arange(nc), nz - 1)
    lay = np.tile(np.arange(nz - 1), nc)
    f = np.arange(nvf)
    rows = np.concatenate([cell(col, lay, nz), cell(col, lay + 1, nz)])
    cols = np.concatenate([f, f])
    vals = np.concatenate([np.ones(nvf), -np.ones(nvf)])
    Dz = sp.csr_matrix((vals, (rows, cols)), shape=(ncells, nvf))

    wc2 = prm.omega_c ** 2
    wn2 = prm.omega_N ** 2
    horiz = Dh @ sp.diags(1.0 / mh) @ Dh.T
    vert = Dz @ sp.diags(1.0 / mz) @ Dz.T
    H = (sp.diags(M3) + wc2 * (horiz + vert / (1.0 + wn2))).tocsr()

    # Delta_h: entries of the horizontal term that couple cells of one column.
    hcoo = horiz.tocoo()
    same_col = (hcoo.row // nz) == (hcoo.col // nz)
    delta_h = sp.csr_matrix((hcoo.data[same_col], (hcoo.row[same_col], hcoo.col[same_col])),
                            shape=(ncells, ncells))
    Hz = (sp.diags(M3) + wc2 * delta_h + (wc2 / (1.0 + wn2)) * vert).tocsr()

    diag = Hz.diagonal().reshape(nc, nz)
    # sub[c, l] = H^_z[(c, l), (c, l-1)]; the entry across a column boundary
    # (l = 0) is zero because H^_z is column block-diagonal.
    sub = np.concatenate([np.zeros(1, dtype=diag.dtype), Hz.diagonal(-1)]).reshape(nc, nz)
    assert np.all(sub[:, 0] == 0)
    op = Operator(nc, nz, M3, Dh, mh, Dz, mz, H, Hz)
    op.Hz_diag = diag
    op.Hz_sub = sub
    return op


def assemble_hierarchy(meshes, prm, theta=None):
    """Operators of all levels (finest first), each rediscretised on its own
    mesh with the finest level's dt (Sec. 3.3 rediscretised coarse operators).

    With theta given on the finest level, level l+1 uses the arithmetic mean
    of theta over the four children of each coarse cell (a reading: the
    paper has no coefficient field).
    """
    ops = []
    th = theta
    for lev, mesh in enumerate(meshes):
        ops.append(assemble(mesh, prm, th))
        if th is not None and lev + 1 < len(meshes):
            nz = prm.nlayers
            th = np.asarray(th).reshape(-1, 4, nz).mean(axis=1).reshape(-1)
    return ops


def apply(op, x):
    """y = H^ x."""
    return op.H @ x


def thomas(sub, diag, sup, rhs):
    """Solve tridiagonal systems by Gaussian elimination without pivoting
    (the Thomas algorithm used at lowest order, Sec. 4.3.1).

    All arrays are (batch, n); sub[:, 0] and sup[:, n-1] are ignored.
    Forward elimination builds the modified super-diagonal cp and right-hand
    side dp; back substitution then recovers x from the last row upwards.
    """
    batch, n = diag.shape
    dtype = np.result_type(sub, diag, sup, rhs)
    cp = np.zeros((batch, n), dtype=dtype)
    dp = np.zeros((batch, n), dtype=dtype)
    denom = diag[:, 0]
    cp[:, 0] = sup[:, 0] / denom if n > 1 else 0.0
    dp[:, 0] = rhs[:, 0] / denom
    for i in range(1, n):
        denom = diag[:, i] - sub[:, i] * cp[:, i - 1]
        if i < n - 1:
            cp[:, i] = sup[:, i] / denom
        dp[:, i] = (rhs[:, i] - sub[:, i] * dp[:, i - 1]) / denom
    x = np.zeros((batch, n), dtype=dtype)
    x[:, n - 1] = dp[:, n - 1]
    for i in range(n - 2, -1, -1):
        x[:, i] = dp[:, i] - cp[:, i] * x[:, i + 1]
    return x


def solve_Hz(op, r):
    """H^_z^-1 r column by column (H^_z is symmetric: super = sub shifted)."""
    nc, nz = op.ncols, op.nlayers
    sub = op.Hz_sub
    sup = np.zeros_like(sub)
    sup[:, :-1] = sub[:, 1:]
    return thomas(sub, op.Hz_diag, sup, np.asarray(r).reshape(nc, nz)).reshape(-1)
