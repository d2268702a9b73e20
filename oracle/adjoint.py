"""Gradients of a least-squares loss of the Helmholtz solution (oracle).

Differentiable form of the solve p = H^(theta)^-1 b, where theta is the
per-cell coefficient dividing each cell's share of the lumped vertical
velocity mass (helmholtz.assemble).  With L = 1/2 ||p - p_t||^2:

    lambda = H^^-T (p - p_t) = H^^-1 (p - p_t)     (H^ is symmetric)
    dL/db = lambda
    dL/dtheta_K = -lambda^T (dH^/dtheta_K) p.

Only the vertical term of Eq. (Preconditioner) depends on theta:
dH^/dtheta_K = w_c^2/(1+w_N^2) D_z diag(d(1/Mz_ff)/dtheta_K) D_z^T, and
d(1/Mz_ff)/dtheta_K = (dz / (3 A_K theta_K^2)) / Mz_ff^2 for the (at most two)
vertical faces f of cell K.  Hence

    dL/dtheta_K = -w_c^2/(1+w_N^2) sum_f (D_z^T lambda)_f (D_z^T p)_f
                  (dz / (3 A_K theta_K^2)) / Mz_ff^2.
"""
import numpy as np

from . import helmholtz


def loss(p, p_target):
    d = p - p_target
    return 0.5 * np.dot(d, d)


def theta_gradient(op, prm, mesh, theta, p, lam):
    """dL/dtheta for the finest-level operator `op` assembled with `theta`."""
    nc, nz = op.ncols, op.nlayers
    wfac = prm.omega_c ** 2 / (1.0 + prm.omega_N ** 2)
    jl = op.Dz.T @ lam            # (D_z^T lambda)_f
    jp = op.Dz.T @ p
    per_face = jl * jp / op.mz ** 2                     # (nc * (nz - 1),)
    area = mesh.area1[:, None] * prm.rho()[None, :] ** 2
    th = np.asarray(theta).reshape(nc, nz)
    dm_dtheta = prm.dz / (3.0 * area * th ** 2)         # -d(Mz share of K)/dtheta_K
    # Scatter: face f touches cells (c, l) and (c, l+1) with D_z entries +1, -1;
    # |D_z|^T maps per-face quantities to the cells on either side.
    per_cell = (abs(op.Dz) @ per_face).reshape(nc, nz)
    return (-wfac * per_cell * dm_dtheta).reshape(-1)


def value_and_grad(ops, prm, mesh, theta, b, p_target, solve):
    """L(theta, b) and its gradients, using `solve(ops, rhs)` for H^^-1."""
    p = solve(ops, b)
    lam = solve(ops, p - p_target)
    return loss(p, p_target), lam, theta_gradient(ops[0], prm, mesh, theta, p, lam), p
