"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds the workload shapes and the random draws only; it contains
none of the solver's arithmetic.  Every vector is drawn on the host in FP64
with ``numpy.random.default_rng(seed)`` so that the CPU oracle and the CUDA
path can be fed bit-identical inputs.

Workloads (the paper's lowest-order grid, Table "Grid setup", is refinement 6
with 64 layers, i.e. 81,920 columns; R = 6371 km, shell thickness 10 km):

    r3x16   refinement 3 x 16 layers,   3 levels, FP64       (smallest case)
    r6x64   refinement 6 x 64 layers,   5 levels, FP64       (paper scale)
    r6x64m  refinement 6 x 64 layers,   5 levels, mixed FP32 cycle / FP64 Krylov
    r5x64a  refinement 5 x 64 layers,   5 levels, FP64, differentiable (theta)
    r7x128  refinement 7 x 128 layers,  6 levels, FP64 and mixed
"""
import numpy as np

WORKLOADS = {
    "r3x16": dict(refinement=3, nlayers=16, nlevels=3, precision="fp64"),
    "r6x64": dict(refinement=6, nlayers=64, nlevels=5, precision="fp64"),
    "r6x64m": dict(refinement=6, nlayers=64, nlevels=5, precision="mixed"),
    "r5x64a": dict(refinement=5, nlayers=64, nlevels=5, precision="fp64", theta=True),
    "r7x128": dict(refinement=7, nlayers=128, nlevels=6, precision="both"),
    # next-to-lowest order (Table "GridSetup"): 5,120 columns x 64 layers, the
    # NLO level plus 4 lowest-order levels (refinements 4 .. 1)
    "r4x64nlo": dict(refinement=4, nlayers=64, nlevels=4, precision="both", order="nlo"),
}

# One seed per independent draw.
SEED_RHS = 0        # right-hand side b ~ N(0, 1) per cell
SEED_PSTAR = 1      # manufactured solution p* ~ N(0, 1)
SEED_THETA = 2      # vertical-coupling coefficient field theta = exp(0.3 N(0,1))
SEED_PTARGET = 3    # adjoint target p_target ~ N(0, 1)
SEED_DIRS = 4       # finite-difference directions
SEED_MIXED = 5      # velocity-pressure right-hand side (R_U, R_P) ~ N(0, 1)
SEED_NLO = 6        # next-to-lowest-order right-hand side ~ N(0, 1) per unknown


def ncolumns(refinement):
    """Number of triangles of an icosahedral mesh refined `refinement` times."""
    return 20 * 4 ** refinement


def ncells(refinement, nlayers):
    return ncolumns(refinement) * nlayers


def normal(n, seed):
    """n iid N(0,1) FP64 samples from the given seed."""
    return np.random.default_rng(seed).standard_normal(n)


def rhs(n, seed=SEED_RHS):
    return normal(n, seed)


def pstar(n, seed=SEED_PSTAR):
    return normal(n, seed)


def theta(n, seed=SEED_THETA, scale=0.3):
    """Log-normal positive coefficient field exp(scale * N(0,1))."""
    return np.exp(scale * normal(n, seed))


def ptarget(n, seed=SEED_PTARGET):
    return normal(n, seed)


def directions(n, count, seed=SEED_DIRS):
    """`count` iid N(0,1) direction vectors of length n, shape (count, n)."""
    return np.random.default_rng(seed).standard_normal((count, n))


def mixed_rhs(nu, np_, seed=SEED_MIXED):
    """Field values (R_U, R_P) of the velocity-pressure right-hand side: nu
    face values, then np_ cell values, iid N(0,1) (faces in face order); the
    system's right-hand side is (M2~ R_U, M3 R_P)."""
    return normal(nu + np_, seed)


def nlo_rhs(n, seed=SEED_NLO):
    """Right-hand side of the next-to-lowest-order Helmholtz problem: n iid
    N(0,1) values, one per DG1 unknown, in the oracle's unknown order."""
    return normal(n, seed)
