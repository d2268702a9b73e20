"""Parity at the full workload sizes, in the configuration bench.py times.

r6x64 (81,920 columns x 64 layers, 5 levels): whole-vector operator and
V-cycle parity, the FP64 solve against the oracle's solve (iteration count
within 1; it is also the count bench.py uses to scale the oracle sample), a
manufactured solution and the mixed form's error.  r5x64 with theta:
adjoint gradients against the oracle and central differences in 32 seeded
directions.  r7x128 (42M cells): the oracle cannot solve it in seconds, so
properties that hold at any size are checked (row sums = cell volumes from
the oracle's mesh, symmetry, converged true residuals, both forms agree).
r4x64 at next-to-lowest order: the same kind of properties.
"""
import numpy as np
import pytest

import bench
import hmg_inputs as gi
from oracle import adjoint, helmholtz, krylov, mesh, multigrid
from tests.helpers import cell_permutation, column_permutation, rel_l2

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1605_00492_gb300 as hmg  # noqa: E402

DEV = "cuda:0"


class Full:
    def __init__(self, name, theta=False, shape=None):
        if shape is None:
            w = gi.WORKLOADS[name]
            self.r, self.nz, self.L = w["refinement"], w["nlayers"], w["nlevels"]
        else:
            self.r, self.nz, self.L = shape
        self.ms = mesh.hierarchy(self.r, self.L)
        self.prm = helmholtz.Params(refinement=self.r, nlayers=self.nz)
        n = self.ms[0].ncols * self.nz
        self.theta = gi.theta(n) if theta else None
        self.ops = helmholtz.assemble_hierarchy(self.ms, self.prm, self.theta)
        self.h = hmg.Hierarchy(self.r, self.nz, self.L)
        cen, _ = self.h.export_mesh(0)
        self.idx = cell_permutation(column_permutation(cen, self.ms[0].centroid), self.nz)
        self.h.assemble(theta=self.gpu(self.theta) if theta else None)

    def gpu(self, v):
        return torch.tensor(np.asarray(v)[self.idx], dtype=torch.float64, device=DEV)

    @staticmethod
    def host(t):
        return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def r6():
    f = Full("r6x64")
    yield f
    f.h.close()


def test_r6x64_apply_and_vcycle(r6):
    x = gi.rhs(r6.ops[0].ncells, seed=7)
    y = r6.h.apply(r6.gpu(x))
    assert rel_l2(r6.host(y), (r6.ops[0].H @ x)[r6.idx]) < 1e-13
    b = gi.rhs(r6.ops[0].ncells)
    z_ref = multigrid.vcycle(r6.ops, b)
    z = r6.h.vcycle(r6.gpu(b))
    assert rel_l2(r6.host(z), z_ref[r6.idx]) < 1e-12
    zm = r6.h.vcycle(r6.gpu(b), precision="mixed")
    assert rel_l2(r6.host(zm), z_ref[r6.idx]) < 1e-4


def test_r6x64_solve_matches_oracle(r6):
    b = gi.rhs(r6.ops[0].ncells)
    x_ref, info_ref = krylov.pcg(r6.ops[0].H.dot, lambda v: multigrid.vcycle(r6.ops, v), b, rtol=1e-8)
    x, info = r6.h.solve(r6.gpu(b), rtol=1e-8)
    assert info["converged"] == 1 and info["true_rel_residual"] < 2e-8
    assert abs(info["iterations"] - info_ref.iterations) <= 1
    assert info_ref.iterations == bench.ORACLE_ITERATIONS
    assert rel_l2(r6.host(x), x_ref[r6.idx]) <= 1e-9
    # mixed form: error against the FP64 oracle solution, stated here
    xm, infom = r6.h.solve(r6.gpu(b), precision="mixed", rtol=1e-8)
    assert infom["converged"] == 1 and infom["true_rel_residual"] < 2e-8
    assert rel_l2(r6.host(xm), x_ref[r6.idx]) < 1e-6


def test_r6x64_manufactured_solution(r6):
    ps = gi.pstar(r6.ops[0].ncells)
    b = r6.ops[0].H @ ps
    x, info = r6.h.solve(r6.gpu(b), rtol=1e-10)
    assert info["converged"] == 1
    assert rel_l2(r6.host(x), ps[r6.idx]) < 1e-6


def test_r5x128_parity_at_128_layers():
    """128 layers per column, as in the r7x128 workload, compared with the
    oracle: refinement 5 (20,480 columns, 640 tiles of 32) x 128 layers
    (2.6 M cells), 5 levels.  The finest level takes the same kernels as
    r7x128's: the FP64 tile sweep with its 66 KB of shared memory (opt-in
    above 48 KB) and, in the mixed form, the FP32 tile sweep (the register
    sweep has no 128-layer variant); level 1 (160 tiles) the staged FP32
    sweep with 115 KB.  The V-cycle tolerances are the 64-layer ones scaled by
    the growth of the column blocks' condition number, which goes as n_z^2
    (about 1.6e3 at 64 layers and 6.4e3 at 128 in the oracle's H^_z blocks of
    this mesh): the split-form smoother of the kernels and the oracle's
    literal form round differently by about eps * kappa(H^_z).  So: operator
    at 1e-13, FP64 V-cycle at 1e-11 (measured 2.8e-12), the mixed V-cycle's
    error against the FP64 oracle V-cycle at 4e-4 (measured 1.0e-4), the FP64
    solve at 1e-9 with the iteration count within 1, and the mixed solve
    against the oracle's FP64 solution (bound 1e-6; measured 8.6e-12)."""
    f = Full(None, shape=(5, 128, 5))
    n = f.ops[0].ncells
    x = gi.rhs(n, seed=7)
    assert rel_l2(f.host(f.h.apply(f.gpu(x))), (f.ops[0].H @ x)[f.idx]) < 1e-13
    b = gi.rhs(n)
    z_ref = multigrid.vcycle(f.ops, b)
    assert rel_l2(f.host(f.h.vcycle(f.gpu(b))), z_ref[f.idx]) < 1e-11
    zm = f.h.vcycle(f.gpu(b), precision="mixed")
    assert rel_l2(f.host(zm), z_ref[f.idx]) < 4e-4
    x_ref, info_ref = krylov.pcg(f.ops[0].H.dot, lambda v: multigrid.vcycle(f.ops, v), b, rtol=1e-8)
    xg, info = f.h.solve(f.gpu(b), rtol=1e-8)
    assert info["converged"] == 1 and abs(info["iterations"] - info_ref.iterations) <= 1
    assert rel_l2(f.host(xg), x_ref[f.idx]) <= 1e-9
    xm, infom = f.h.solve(f.gpu(b), precision="mixed", rtol=1e-8)
    assert infom["converged"] == 1 and infom["true_rel_residual"] < 2e-8
    assert rel_l2(f.host(xm), x_ref[f.idx]) < 1e-6
    f.h.close()


def test_r5x64_adjoint_gradients():
    f = Full("r5x64a", theta=True)
    n = f.ops[0].ncells
    kw = dict(rtol=1e-13, max_iter=400)
    b = f.gpu(gi.rhs(n)).requires_grad_(True)
    th = f.gpu(f.theta).requires_grad_(True)
    p = hmg.HelmholtzSolve.apply(f.h, b, th, kw, kw)
    pt = f.gpu(gi.ptarget(n)) * p.detach().abs().max()
    loss = 0.5 * ((p - pt) ** 2).sum()
    loss.backward()
    solve = lambda ops, rhs: krylov.pcg(ops[0].H.dot, lambda v: multigrid.vcycle(ops, v), rhs, rtol=1e-13,
                                        max_iter=400)[0]
    pt_or = np.empty(n)
    pt_or[f.idx] = f.host(pt)
    L_ref, lam_ref, g_ref, _ = adjoint.value_and_grad(f.ops, f.prm, f.ms[0], f.theta, gi.rhs(n), pt_or, solve)
    assert float(loss.detach()) == pytest.approx(L_ref, rel=1e-9)
    assert rel_l2(f.host(b.grad), lam_ref[f.idx]) < 1e-8
    assert rel_l2(f.host(th.grad), g_ref[f.idx]) < 1e-8
    # central differences, h = 1e-6, 32 seeded directions
    with torch.no_grad():
        for v in gi.directions(n, 32):
            vg = f.gpu(v)
            Lp = 0.5 * ((hmg.HelmholtzSolve.apply(f.h, b, th + 1e-6 * vg, kw, kw) - pt) ** 2).sum()
            Lm = 0.5 * ((hmg.HelmholtzSolve.apply(f.h, b, th - 1e-6 * vg, kw, kw) - pt) ** 2).sum()
            fd = float(Lp - Lm) / 2e-6
            assert float((th.grad * vg).sum()) == pytest.approx(fd, rel=1e-5)
    f.h.close()


def test_r7x128_properties_both_forms():
    w = gi.WORKLOADS["r7x128"]
    r, nz, L = w["refinement"], w["nlayers"], w["nlevels"]
    m = mesh.hierarchy(r, 1)[0]
    prm = helmholtz.Params(refinement=r, nlayers=nz)
    vol = (m.area1[:, None] * prm.rho()[None, :] ** 2 * prm.dz).reshape(-1)
    h = hmg.Hierarchy(r, nz, L)
    h.assemble()
    cen, _ = h.export_mesh(0)
    idx = cell_permutation(column_permutation(cen, m.centroid), nz)
    n = h.ncells
    ones = torch.ones(n, dtype=torch.float64, device=DEV)
    y = h.apply(ones).cpu().numpy()
    # the diagonal (~1e16) cancels against the vertical couplings to ~1e11: rounding ~1e-10 relative
    assert np.max(np.abs(y - vol[idx]) / vol[idx]) < 1e-8
    x1 = torch.tensor(gi.rhs(n, seed=8), device=DEV)
    x2 = torch.tensor(gi.rhs(n, seed=9), device=DEV)
    a = float(torch.dot(x1, h.apply(x2)))
    c = float(torch.dot(x2, h.apply(x1)))
    assert a == pytest.approx(c, rel=1e-12)
    b = torch.tensor(gi.rhs(n), device=DEV)
    x64, i64 = h.solve(b, rtol=1e-8)
    xm, im = h.solve(b, precision="mixed", rtol=1e-8)
    assert i64["converged"] == 1 and im["converged"] == 1
    assert i64["true_rel_residual"] < 2e-8 and im["true_rel_residual"] < 2e-8
    assert float(torch.linalg.norm(xm - x64) / torch.linalg.norm(x64)) < 1e-6
    h.close()


def test_velocity_pressure_system_full_size():
    """r6x64 (18.3 M unknowns): GMRES(30) with the Schur-complement
    preconditioner converges with both V-cycle forms to the same solution; the
    operator's off-diagonal blocks are adjoint (<D U, P> = <U, D^T P>) and its
    velocity mass is symmetric, properties that hold at any size."""
    h = hmg.Hierarchy(6, 64, 5)
    h.assemble()
    nhf, nvf, nc = h.mixed_sizes()
    nu = nhf + nvf
    g = torch.Generator(device=DEV).manual_seed(17)
    U1 = torch.randn(nu, generator=g, dtype=torch.float64, device=DEV)
    U2 = torch.randn(nu, generator=g, dtype=torch.float64, device=DEV)
    P = torch.randn(nc, generator=g, dtype=torch.float64, device=DEV)
    zu, zp = torch.zeros(nu, dtype=torch.float64, device=DEV), torch.zeros(nc, dtype=torch.float64, device=DEV)
    yu_p, _ = h.mixed_apply(zu, P)            # -a D^T P
    _, yp_u = h.mixed_apply(U1, zp)           # a c^2 D U
    a_c2_over_minus_a = float(torch.dot(yp_u, P)) / float(torch.dot(U1, yu_p))   # = -c^2
    assert a_c2_over_minus_a == pytest.approx(-300.0 ** 2, rel=1e-10)
    m1, _ = h.mixed_apply(U1, zp)
    m2, _ = h.mixed_apply(U2, zp)
    assert float(torch.dot(m1, U2)) == pytest.approx(float(torch.dot(U1, m2)), rel=1e-12)
    # right-hand side (M2~ R_U, M3 R_P)
    R = torch.tensor(gi.mixed_rhs(nu, nc), dtype=torch.float64, device=DEV)
    bu, _ = h.mixed_apply(R[:nu].contiguous(), zp)
    _, bp = h.mixed_apply(zu, R[nu:].contiguous())
    u64, p64, i64 = h.mixed_solve(bu, bp, rtol=1e-8)
    um, pm, im = h.mixed_solve(bu, bp, rtol=1e-8, precision="mixed")
    assert i64["converged"] == 1 and im["converged"] == 1
    assert i64["true_rel_residual"] < 2e-8 and im["true_rel_residual"] < 2e-8
    assert float(torch.linalg.norm(um - u64) / torch.linalg.norm(u64)) < 1e-6
    assert float(torch.linalg.norm(pm - p64) / torch.linalg.norm(p64)) < 1e-6
    h.close()


def test_nlo_full_size_properties():
    """r4x64 at next-to-lowest order (Table "GridSetup": 5,120 columns x 64
    layers, 2.0 M pressure unknowns): the oracle cannot assemble and solve it
    in seconds, so properties that hold at any size are checked: H^ is
    symmetric; H^ 1 = M3 1 = |K| / 6 per unknown, with |K| = A_T(rho_l) dz
    from the flat triangles of the exported vertices; the V-cycle is symmetric
    and positive; both V-cycle forms converge to the same solution."""
    w = gi.WORKLOADS["r4x64nlo"]
    r, nz = w["refinement"], w["nlayers"]
    h = hmg.Hierarchy(r, nz, w["nlevels"])
    h.assemble()
    n = h.nlo_size()
    g = torch.Generator(device=DEV).manual_seed(23)
    x = torch.randn(n, generator=g, dtype=torch.float64, device=DEV)
    y = torch.randn(n, generator=g, dtype=torch.float64, device=DEV)
    xHy, yHx = float(torch.dot(x, h.nlo_apply(y))), float(torch.dot(y, h.nlo_apply(x)))
    assert xHy == pytest.approx(yHx, rel=1e-12)
    V = h.export_vertices(0)
    A1 = 0.5 * np.linalg.norm(np.cross(V[:, 1] - V[:, 0], V[:, 2] - V[:, 0]), axis=1)
    prm = helmholtz.Params(refinement=r, nlayers=nz)
    vol = A1[:, None] * prm.rho()[None, :] ** 2 * prm.dz
    ones = torch.ones(n, dtype=torch.float64, device=DEV)
    got = h.nlo_apply(ones).cpu().numpy().reshape(-1, nz, 6)
    assert np.allclose(got, vol[:, :, None] / 6.0, rtol=1e-8)
    Vx, Vy = h.nlo_vcycle(x), h.nlo_vcycle(y)
    assert float(torch.dot(Vx, y)) == pytest.approx(float(torch.dot(x, Vy)), rel=1e-10)
    assert float(torch.dot(x, Vx)) > 0
    b = torch.tensor(gi.nlo_rhs(n), dtype=torch.float64, device=DEV)
    x64, i64 = h.nlo_solve(b, rtol=1e-8)
    xm, im = h.nlo_solve(b, rtol=1e-8, precision="mixed")
    assert i64["converged"] == 1 and im["converged"] == 1
    assert i64["true_rel_residual"] < 2e-8 and im["true_rel_residual"] < 2e-8
    assert i64["iterations"] <= 40
    assert float(torch.linalg.norm(xm - x64) / torch.linalg.norm(x64)) < 1e-6
    h.close()


def test_nlo_velocity_pressure_system_full_size():
    """r4x64 at NLO (Table "GridSetup": 7.9 M unknowns; 7,848,960 here): the off-diagonal
    blocks are adjoint up to the factor -c^2 (<D U, P> = <U, D^T P>), the
    velocity mass is symmetric, and GMRES with the Schur-complement
    preconditioner converges with both V-cycle forms to the same solution."""
    w = gi.WORKLOADS["r4x64nlo"]
    h = hmg.Hierarchy(w["refinement"], w["nlayers"], w["nlevels"])
    h.assemble()
    sizes = h.nlo_mixed_sizes()
    n = sum(sizes)
    nu = n - sizes[3]
    # Table "GridSetup" counts 24 per cell, one boundary node of vertical
    # velocity per column and vertex included (top and bottom carry none here)
    assert n == 24 * 5120 * 64 - 3 * 5120 and round((n + 3 * 5120) / 1e6, 1) == 7.9
    g = torch.Generator(device=DEV).manual_seed(29)
    rnd = lambda: torch.randn(n, generator=g, dtype=torch.float64, device=DEV)
    U1, U2, P = rnd(), rnd(), rnd()
    U1[nu:] = 0
    U2[nu:] = 0
    P[:nu] = 0
    yP = h.nlo_mixed_apply(P)          # (-a D^T P, M3 P)
    yU = h.nlo_mixed_apply(U1)         # (M2~ U1, a c^2 D U1)
    ratio = float(torch.dot(yU[nu:], P[nu:])) / float(torch.dot(U1[:nu], yP[:nu]))
    assert ratio == pytest.approx(-300.0 ** 2, rel=1e-10)
    yU2 = h.nlo_mixed_apply(U2)
    assert float(torch.dot(yU[:nu], U2[:nu])) == pytest.approx(float(torch.dot(U1[:nu], yU2[:nu])), rel=1e-12)
    R = torch.tensor(gi.mixed_rhs(nu, sizes[3]), dtype=torch.float64, device=DEV)
    Ru, Rp = R.clone(), R.clone()
    Ru[nu:] = 0
    Rp[:nu] = 0
    b = torch.cat([h.nlo_mixed_apply(Ru)[:nu], h.nlo_mixed_apply(Rp)[nu:]])
    x64, i64 = h.nlo_mixed_solve(b, rtol=1e-10, max_iter=500)
    xm, im = h.nlo_mixed_solve(b, rtol=1e-10, precision="mixed", max_iter=500)
    assert i64["converged"] == 1 and im["converged"] == 1
    assert i64["true_rel_residual"] < 2e-10 and im["true_rel_residual"] < 2e-10
    for sl in (slice(0, nu), slice(nu, n)):
        assert float(torch.linalg.norm(xm[sl] - x64[sl]) / torch.linalg.norm(x64[sl])) < 1e-7
    _, i5 = h.nlo_mixed_solve(b, rtol=1e-5)
    assert i5["iterations"] <= 30
    h.close()
