"""Outer Krylov solves of H^ p = b preconditioned by the V-cycle (oracle).

The paper wraps the multigrid preconditioner in restarted GMRES(30) on the
mixed system (Sec. 5) and notes that CG is the method of choice when the
operator is symmetric positive definite, which H^ is.  Here:

* ``pcg``   textbook preconditioned conjugate gradients, x0 = 0, stopped when
            ||r_k||_2 / ||r_0||_2 < rtol with the recursively updated residual;
* ``fpcg``  flexible CG (Polak-Ribiere beta = z_k.(r_k - r_k-1) / z_k-1.r_k-1)
            for a preconditioner that is not exactly linear or symmetric
            (the FP32 V-cycle of the mixed-precision form);
* ``fgmres`` restarted GMRES(m) with the preconditioner on the right, in its
            flexible form (the preconditioned directions z_j are kept, so the
            V-cycle may vary between steps): Arnoldi with modified
            Gram-Schmidt, Givens rotations on the Hessenberg matrix, and the
            least-squares residual |g_(j+1)| / ||r_0|| as the stopping test
            (Saad, Iterative Methods for Sparse Linear Systems, 2nd ed.,
            Sec. 6.5 and Algorithm 9.6).  The iterate is formed at the end of
            every restart cycle and at convergence; the residual that starts a
            cycle is recomputed from it, b - A x.
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


def fgmres(apply_A, precond, b, rtol=1e-8, max_iter=500, restart=30):
    info = SolveInfo()
    x = np.zeros_like(b)
    r0 = np.linalg.norm(b)
    info.residuals.append(1.0)
    if r0 == 0.0:
        info.converged = True
        return x, info
    m = restart
    k = 0
    r = b.copy()
    while k < max_iter:
        beta = np.linalg.norm(r)
        V = np.zeros((m + 1, b.size))
        Z = np.zeros((m, b.size))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_end = 0
        for j in range(m):
            Z[j] = precond(V[j])
            w = apply_A(Z[j])
            for i in range(j + 1):               # modified Gram-Schmidt
                H[i, j] = np.dot(w, V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):                   # earlier rotations on column j
                a, c = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * a + sn[i] * c
                H[i + 1, j] = -sn[i] * a + cs[i] * c
            den = np.hypot(H[j, j], H[j + 1, j])  # rotation that zeroes H[j+1, j]
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k += 1
            j_end = j + 1
            rel = abs(g[j + 1]) / r0
            info.residuals.append(rel)
            info.iterations = k
            if rel < rtol or k >= max_iter:
                break
        # y = R^-1 g by back substitution; x += Z y
        y = np.zeros(j_end)
        for i in range(j_end - 1, -1, -1):
            y[i] = (g[i] - np.dot(H[i, i + 1:j_end], y[i + 1:j_end])) / H[i, i]
        x = x + Z[:j_end].T @ y
        if info.residuals[-1] < rtol:
            info.converged = True
            break
        r = b - apply_A(x)
    return x, info
