"""Tensor-product (horizontal-only) geometric multigrid V-cycle (oracle).

* Smoother: block-Jacobi vertical line relaxation, Eq. (BlockJacobi) in the
  form of the operator split of Sec. 5.4 ("smoother application"):
      u <- u + omega H^_z^-1 (b - H^ u),  omega = 0.8 (Sec. 5).
  (Eq. BlockJacobi as printed reads P -> P + omega H^_z^-1 (P - H^ R_p);
  the symbols there are garbled, and the smoother-application formula of
  Sec. 5.4 is the one used.)
* Transfers: DG0 spaces on nested meshes (Sec. 3.2); prolongation is the
  natural embedding, i.e. the coarse value copied to the 4 children in every
  layer (columns are kept intact: horizontal semi-coarsening, Sec. 4.2.1);
  the residual is a dual (assembled) vector, so it is restricted with the
  transpose, i.e. summed over the 4 children.
* Cycle: the correction scheme of Algorithm 1 applied recursively, with
  nu_pre pre- and nu_post post-smoothing steps per level and n_coarse
  smoother iterations from a zero guess on the coarsest level (Sec. 5: "two
  smoother iterations").
"""
import numpy as np
import scipy.sparse as sp

from . import helmholtz


def smooth(op, u, b, omega):
    """One block-Jacobi line-relaxation step u + omega H^_z^-1 (b - H^ u)."""
    return u + omega * helmholtz.solve_Hz(op, b - op.H @ u)


def prolongation(ncols_coarse, nlayers):
    """P: coarse DG0 vector -> fine DG0 vector; fine column f gets the value of
    coarse column f // 4 in the same layer.  Shape (4 ncols_c nz, ncols_c nz)."""
    nf = 4 * ncols_coarse
    fine_cells = np.arange(nf * nlayers)
    fine_col = fine_cells // nlayers
    layer = fine_cells % nlayers
    coarse_cells = (fine_col // 4) * nlayers + layer
    return sp.csr_matrix((np.ones(nf * nlayers), (fine_cells, coarse_cells)),
                         shape=(nf * nlayers, ncols_coarse * nlayers))


def prolong(e_coarse, ncols_coarse, nlayers):
    return prolongation(ncols_coarse, nlayers) @ e_coarse


def restrict(r_fine, ncols_coarse, nlayers):
    return prolongation(ncols_coarse, nlayers).T @ r_fine


def vcycle(ops, b, omega=0.8, nu_pre=2, nu_post=2, n_coarse=2, level=0):
    """Approximate H^_level^-1 b by one V-cycle from a zero initial guess."""
    op = ops[level]
    u = np.zeros_like(b)
    if level == len(ops) - 1:
        for _ in range(n_coarse):
            u = smooth(op, u, b, omega)
        return u
    for _ in range(nu_pre):                                  # presmooth (M1)
        u = smooth(op, u, b, omega)
    nc_coarse = ops[level + 1].ncols
    b_c = restrict(b - op.H @ u, nc_coarse, op.nlayers)      # restrict residual (M2)
    e_c = vcycle(ops, b_c, omega, nu_pre, nu_post, n_coarse, level + 1)   # (M3)
    u = u + prolong(e_c, nc_coarse, op.nlayers)              # prolong correction (M4)
    for _ in range(nu_post):                                 # postsmooth (M5)
        u = smooth(op, u, b, omega)
    return u
