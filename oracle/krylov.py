"""Outer Krylov solves of H^ p = b preconditioned by the V-cycle (oracle).

The paper wraps the multigrid preconditioner in restarted GMRES(30) on the
mixed system (Sec. 5) and notes that CG is the method of choice when the
operator is symmetric positive definite, which H^ is.  Here:

* ``pcg``   textbook preconditioned conjugate gradients, x0 = 0, stopped when
            ||r_k||_2 / ||r_0||_2 < rtol with the recursively updated residual;
* ``fpcg``  flexible CG (Polak-Ribiere beta = z_k.(r_k - r_k-1) / z_k-1.r_k-1)
            for a preconditioner that is not exactly linear or symmetric
            (the FP32 V-cycle of the mixed-precision form).
"""
import numpy as np


class SolveInfo:
    def __init__(self):
        self.iterations = 0
        self.residuals = []     # ||r_k|| / ||r_0||, k = 0, 1, ...
        self.converged = False

    def __repr__(self):
        return f"SolveInfo(iterations={self.iterations}, converged={self.converged}, rel={self.residuals[-1]:.3e})"


def pcg(apply_A, precond, b, rtol=1e-8, max_iter=500):
    info = SolveInfo()
    x = np.zeros_like(b)
    r = b.copy()
    r0 = np.linalg.norm(r)
    info.residuals.append(1.0)
    if r0 == 0.0:
        info.converged = True
        return x, info
    z = precond(r)
    p = z.copy()
    rz = np.dot(r, z)
    for k in range(1, max_iter + 1):
        q = apply_A(p)
        alpha = rz / np.dot(p, q)
        x = x + alpha * p
        r = r - alpha * q
        rel = np.linalg.norm(r) / r0
        info.residuals.append(rel)
        info.iterations = k
        if rel < rtol:
            info.converged = True
            break
        z = precond(r)
        rz_new = np.dot(r, z)
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    return x, info


def fpcg(apply_A, precond, b, rtol=1e-8, max_iter=500):
    info = SolveInfo()
    x = np.zeros_like(b)
    r = b.copy()
    r0 = np.linalg.norm(r)
    info.residuals.append(1.0)
    if r0 == 0.0:
        info.converged = True
        return x, info
    z = precond(r)
    p = z.copy()
    rz = np.dot(r, z)
    r_old = r
    for k in range(1, max_iter + 1):
        q = apply_A(p)
        alpha = rz / np.dot(p, q)
        x = x + alpha * p
        r_old = r
        r = r - alpha * q
        rel = np.linalg.norm(r) / r0
        info.residuals.append(rel)
        info.iterations = k
        if rel < rtol:
            info.converged = True
            break
        z = precond(r)
        beta = np.dot(z, r - r_old) / rz
        rz = np.dot(r, z)
        p = z + beta * p
    return x, info
