"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on
identical seeded inputs.  Cells are matched by column centroid.

Tolerances (FP64): operator application 1e-13 relative L2 (one rounding per
term, no cancellation for random x); fixed-iteration V-cycles 1e-12 (the
split-form smoother of the kernels and the literal form of the oracle differ
by rounding only); solves 1e-9 relative L2 with the iteration count within 1
(the contract of the FP64 method).  FP32 (mixed form) results are compared
against the FP64 oracle with the error stated in each test.
"""
import numpy as np
import pytest

import hmg_inputs as gi
from oracle import adjoint, helmholtz, krylov, mesh, multigrid
from tests.helpers import cell_permutation, column_permutation, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU, skipped there
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1605_00492_gb300 as hmg  # noqa: E402

DEV = "cuda:0"


class Case:
    """One workload on both sides, with the GPU <- oracle cell map."""

    def __init__(self, r, nz, L, theta_seed=None, **op):
        self.r, self.nz, self.L = r, nz, L
        self.ms = mesh.hierarchy(r, L)
        self.prm = helmholtz.Params(refinement=r, nlayers=nz, **op)
        n = self.ms[0].ncols * nz
        self.theta = gi.theta(n, seed=theta_seed) if theta_seed is not None else None
        self.ops = helmholtz.assemble_hierarchy(self.ms, self.prm, self.theta)
        self.h = hmg.Hierarchy(r, nz, L)
        self.idx = []
        for lev in range(L):
            cen, nbr = self.h.export_mesh(lev)
            perm = column_permutation(cen, self.ms[lev].centroid)
            # neighbour tables agree under the permutation
            assert np.all(np.sort(perm[nbr], 1) == np.sort(self.ms[lev].nbr[perm], 1))
            self.idx.append(cell_permutation(perm, nz))
        th = self.gpu(self.theta) if self.theta is not None else None
        opk = {k: v for k, v in op.items() if k in ("c", "N", "nu_cfl", "omega")}
        self.h.assemble(theta=th, **opk)

    def gpu(self, v, level=0):
        return torch.tensor(np.asarray(v)[self.idx[level]], dtype=torch.float64, device=DEV)

    def host(self, t):
        return t.detach().cpu().numpy().astype(np.float64)

    def oracle_order(self, v_gpu, level=0):
        out = np.empty_like(v_gpu)
        out[self.idx[level]] = v_gpu
        return out


_CACHE = {}


def case(*args, **kw):
    key = (args, tuple(sorted(kw.items())))
    if key not in _CACHE:
        _CACHE[key] = Case(*args, **kw)
    return _CACHE[key]


# --------------------------------------------------------------- operator

@pytest.mark.parametrize("r,nz,L", [(0, 1, 1), (1, 4, 2), (3, 16, 3), (2, 7, 3)])
def test_apply_fp64_every_level(r, nz, L):
    c = case(r, nz, L)
    rng = np.random.default_rng(11)
    for lev in range(L):
        x = rng.standard_normal(c.ops[lev].ncells)
        y_ref = c.ops[lev].H @ x
        y = c.h.apply(c.gpu(x, lev), level=lev)
        assert rel_l2(c.host(y), y_ref[c.idx[lev]]) < 1e-13


def test_apply_row_sums_are_cell_volumes():
    c = case(3, 16, 3)
    y = c.host(c.h.apply(torch.ones(c.ops[0].ncells, dtype=torch.float64, device=DEV)))
    vol = c.ops[0].M3[c.idx[0]]
    diag = c.ops[0].H.diagonal()[c.idx[0]]
    assert np.max(np.abs(y - vol) / diag) < 1e-14


def test_apply_fp32_and_tiled_layout():
    c = case(3, 16, 3)
    x = gi.rhs(c.ops[0].ncells, seed=5)
    y_ref = (c.ops[0].H @ x)[c.idx[0]]
    xg = c.gpu(x)
    y32 = c.h.apply(xg.float())
    assert rel_l2(c.host(y32), y_ref) < 2e-6
    xt = c.h.to_layout(xg, "column", "tiled")
    yt = c.h.apply(xt, layout="tiled")
    y = c.h.to_layout(yt, "tiled", "column")
    assert rel_l2(c.host(y), y_ref) < 1e-13
    # padding entries of the tiled layout stay zero
    info = c.h.levels[0]
    assert yt.numel() == info["ncells_padded"]


def test_theta_operator():
    c = case(2, 8, 2, theta_seed=gi.SEED_THETA)
    rng = np.random.default_rng(3)
    for lev in range(2):
        x = rng.standard_normal(c.ops[lev].ncells)
        y = c.h.apply(c.gpu(x, lev), level=lev)
        assert rel_l2(c.host(y), (c.ops[lev].H @ x)[c.idx[lev]]) < 1e-13


# --------------------------------------------------------------- V-cycle

@pytest.mark.parametrize("r,nz,L,nu,nc", [(3, 16, 3, 2, 2), (3, 16, 3, 1, 2), (1, 4, 2, 2, 3), (4, 8, 3, 2, 1),
                                          (2, 5, 1, 2, 2)])
def test_vcycle_fp64(r, nz, L, nu, nc):
    c = case(r, nz, L)
    b = gi.rhs(c.ops[0].ncells)
    z_ref = multigrid.vcycle(c.ops, b, nu_pre=nu, nu_post=nu, n_coarse=nc)
    z = c.h.vcycle(c.gpu(b), nu_pre=nu, nu_post=nu, n_coarse=nc)
    assert rel_l2(c.host(z), z_ref[c.idx[0]]) < 1e-12


def test_vcycle_mixed_against_fp64_oracle():
    c = case(3, 16, 3)
    b = gi.rhs(c.ops[0].ncells)
    z_ref = multigrid.vcycle(c.ops, b)
    z = c.h.vcycle(c.gpu(b), precision="mixed")
    err = rel_l2(c.host(z), z_ref[c.idx[0]])
    assert err < 1e-4, err


def test_vcycle_is_deterministic():
    c = case(3, 16, 3)
    b = c.gpu(gi.rhs(c.ops[0].ncells))
    z1 = c.h.vcycle(b)
    z2 = c.h.vcycle(b)
    assert torch.equal(z1, z2)


# --------------------------------------------------------------- solve

@pytest.mark.parametrize("r,nz,L", [(3, 16, 3), (4, 16, 4), (2, 8, 1), (3, 1, 3)])
def test_solve_fp64_matches_oracle(r, nz, L):
    c = case(r, nz, L)
    b = gi.rhs(c.ops[0].ncells)
    x_ref, info_ref = krylov.pcg(c.ops[0].H.dot, lambda v: multigrid.vcycle(c.ops, v), b, rtol=1e-8,
                                 max_iter=500)
    x, info = c.h.solve(c.gpu(b), rtol=1e-8)
    assert info["converged"] == 1
    assert abs(info["iterations"] - info_ref.iterations) <= 1, (info, info_ref.iterations)
    assert rel_l2(c.host(x), x_ref[c.idx[0]]) <= 1e-9
    assert info["true_rel_residual"] < 2e-8


def test_solve_manufactured_solution():
    c = case(3, 16, 3)
    ps = gi.pstar(c.ops[0].ncells)
    b = c.ops[0].H @ ps
    x, info = c.h.solve(c.gpu(b), rtol=1e-10)
    assert rel_l2(c.host(x), ps[c.idx[0]]) < 1e-7


def test_solve_mixed_precision_error_against_oracle():
    c = case(3, 16, 3)
    b = gi.rhs(c.ops[0].ncells)
    x_ref, _ = krylov.pcg(c.ops[0].H.dot, lambda v: multigrid.vcycle(c.ops, v), b, rtol=1e-12)
    x, info = c.h.solve(c.gpu(b), precision="mixed", rtol=1e-8)
    assert info["converged"] == 1 and info["true_rel_residual"] < 2e-8
    assert rel_l2(c.host(x), x_ref[c.idx[0]]) < 1e-6


@pytest.mark.parametrize("nz", [16, 32])
def test_mixed_on_register_sweep_levels(nz):
    # 20,480 columns = 640 tiles: the FP32 cycle's finest level takes the
    # register-resident sweep and residual, the final sweep carrying the dots.
    c = case(5, nz, 3)
    b = gi.rhs(c.ops[0].ncells)
    z_ref = multigrid.vcycle(c.ops, b)
    z = c.h.vcycle(c.gpu(b), precision="mixed")
    assert rel_l2(c.host(z), z_ref[c.idx[0]]) < 1e-4
    x_ref, _ = krylov.pcg(c.ops[0].H.dot, lambda v: multigrid.vcycle(c.ops, v), b, rtol=1e-12)
    for kind in ("cg", "fcg", "gmres"):
        x, info = c.h.solve(c.gpu(b), precision="mixed", krylov=kind, rtol=1e-8)
        assert info["converged"] == 1 and info["true_rel_residual"] < 2e-8, (kind, info)
        assert rel_l2(c.host(x), x_ref[c.idx[0]]) < 1e-6, kind


def test_solve_flexible_cg_fp64():
    c = case(3, 16, 3)
    b = gi.rhs(c.ops[0].ncells)
    x_ref, info_ref = krylov.fpcg(c.ops[0].H.dot, lambda v: multigrid.vcycle(c.ops, v), b, rtol=1e-8)
    x, info = c.h.solve(c.gpu(b), krylov="fcg", rtol=1e-8)
    assert abs(info["iterations"] - info_ref.iterations) <= 1
    assert rel_l2(c.host(x), x_ref[c.idx[0]]) <= 1e-9


@pytest.mark.parametrize("restart,orth", [(30, 1), (30, 2), (4, 1), (4, 2), (1, 1)])
def test_solve_gmres_fp64_matches_oracle(restart, orth):
    c = case(3, 16, 3)
    b = gi.rhs(c.ops[0].ncells)
    x_ref, info_ref = krylov.fgmres(c.ops[0].H.dot, lambda v: multigrid.vcycle(c.ops, v), b, rtol=1e-8,
                                    restart=restart)
    x, info = c.h.solve(c.gpu(b), krylov="gmres", restart=restart, rtol=1e-8, orth=orth)
    assert info["converged"] == 1 and info["true_rel_residual"] < 2e-8
    assert abs(info["iterations"] - info_ref.iterations) <= 1, (info, info_ref.iterations)
    assert info["rel_residual"] == pytest.approx(info_ref.residuals[-1], rel=1e-3)
    assert rel_l2(c.host(x), x_ref[c.idx[0]]) <= 1e-9


def test_solve_gmres_fixed_steps_match_oracle_iterate():
    """A fixed number of Arnoldi steps with no stopping (rtol tiny): the
    iterate after 5 steps of GMRES(3) (a restart inside) against the
    oracle's, element by element."""
    c = case(2, 8, 2)
    b = gi.rhs(c.ops[0].ncells)
    x_ref, _ = krylov.fgmres(c.ops[0].H.dot, lambda v: multigrid.vcycle(c.ops, v), b, rtol=1e-300,
                             max_iter=5, restart=3)
    x, info = c.h.solve(c.gpu(b), krylov="gmres", restart=3, rtol=1e-300, max_iter=5, raise_on_failure=False)
    assert info["status"] == "HMG_ERR_NOT_CONVERGED" and info["iterations"] == 5
    assert rel_l2(c.host(x), x_ref[c.idx[0]]) <= 1e-10


def test_solve_gmres_mixed_and_status_codes():
    c = case(3, 16, 3)
    b = gi.rhs(c.ops[0].ncells)
    x_ref, _ = krylov.pcg(c.ops[0].H.dot, lambda v: multigrid.vcycle(c.ops, v), b, rtol=1e-12)
    x, info = c.h.solve(c.gpu(b), precision="mixed", krylov="gmres", rtol=1e-8)
    assert info["converged"] == 1 and info["true_rel_residual"] < 2e-8
    assert rel_l2(c.host(x), x_ref[c.idx[0]]) < 1e-6
    for bad in (0, 33):
        with pytest.raises(hmg.HMGError) as e:
            c.h.solve(c.gpu(b), krylov="gmres", restart=bad)
        assert e.value.name == "HMG_ERR_INVALID_ARG"
    bn = b.copy()
    bn[5] = np.inf
    _, info = c.h.solve(c.gpu(bn), krylov="gmres", raise_on_failure=False)
    assert info["status"] == "HMG_ERR_NONFINITE"
    x, info = c.h.solve(torch.zeros(c.ops[0].ncells, dtype=torch.float64, device=DEV), krylov="gmres")
    assert info["converged"] == 1 and torch.count_nonzero(x) == 0
    # a longer restart reallocates the basis; the solve after it still agrees
    x2, _ = c.h.solve(c.gpu(b), krylov="gmres", restart=32, rtol=1e-8)
    x3, _ = c.h.solve(c.gpu(b), krylov="gmres", restart=30, rtol=1e-8)
    assert torch.equal(x2, x3)


@pytest.mark.parametrize("krylov_kind", ["cg", "gmres"])
def test_single_level_method_matches_oracle(krylov_kind):
    """levels=1: two block-Jacobi vertical line relaxations as the
    preconditioner (the single-level method of Sec. 6) on a 3-level context."""
    c = case(3, 16, 3)
    b = gi.rhs(c.ops[0].ncells)
    P = lambda v: multigrid.vcycle(c.ops[:1], v)
    solver = krylov.pcg if krylov_kind == "cg" else krylov.fgmres
    x_ref, info_ref = solver(c.ops[0].H.dot, P, b, rtol=1e-8, max_iter=500)
    x, info = c.h.solve(c.gpu(b), krylov=krylov_kind, levels=1, rtol=1e-8, max_iter=500)
    assert info["converged"] == 1
    assert abs(info["iterations"] - info_ref.iterations) <= 1, (info, info_ref.iterations)
    assert rel_l2(c.host(x), x_ref[c.idx[0]]) <= 1e-9
    _, info_mg = c.h.solve(c.gpu(b), krylov=krylov_kind, rtol=1e-8)
    assert info["iterations"] > 2 * info_mg["iterations"]
    with pytest.raises(hmg.HMGError):
        c.h.solve(c.gpu(b), levels=4)


@pytest.mark.parametrize("pin_b,pin_x", [(True, True), (False, False), (True, False), (False, True)])
def test_solve_host_buffers(pin_b, pin_x):
    """Page-locked buffers are read and written in place by the layout
    kernels, pageable ones go through copies: the same solution either way."""
    c = case(3, 16, 3)
    b = gi.rhs(c.ops[0].ncells)[c.idx[0]]
    bh = torch.tensor(b, dtype=torch.float64)
    xh = torch.full_like(bh, np.nan)
    if pin_b:
        bh = bh.pin_memory()
    if pin_x:
        xh = xh.pin_memory()
    xd, _ = c.h.solve(torch.tensor(b, device=DEV))
    c.h.solve_host(bh, xh)
    assert torch.equal(xh, xd.cpu())


def test_solve_status_codes():
    c = case(2, 8, 2)
    b = gi.rhs(c.ops[0].ncells)
    x, info = c.h.solve(c.gpu(b), max_iter=1, raise_on_failure=False)
    assert info["status"] == "HMG_ERR_NOT_CONVERGED" and info["iterations"] == 1
    bn = b.copy()
    bn[17] = np.nan
    _, info = c.h.solve(c.gpu(bn), raise_on_failure=False)
    assert info["status"] == "HMG_ERR_NONFINITE"
    x, info = c.h.solve(torch.zeros(c.ops[0].ncells, dtype=torch.float64, device=DEV))
    assert info["converged"] == 1 and torch.count_nonzero(x) == 0
    with pytest.raises(hmg.HMGError) as e:
        c.h.solve(c.gpu(b), rtol=2.0)
    assert e.value.name == "HMG_ERR_INVALID_ARG"
    fresh = hmg.Hierarchy(1, 2, 1)
    with pytest.raises(hmg.HMGError) as e:
        fresh.solve(torch.ones(fresh.ncells, dtype=torch.float64, device=DEV))
    assert e.value.name == "HMG_ERR_STATE"
    # the context stays usable after the errors
    _, info = c.h.solve(c.gpu(b))
    assert info["converged"] == 1


# --------------------------------------------------------------- adjoint

def test_theta_gradient_matches_oracle():
    c = case(2, 8, 2, theta_seed=gi.SEED_THETA)
    n = c.ops[0].ncells
    b = gi.rhs(n)
    pt = gi.ptarget(n)
    p = np.asarray(krylov.pcg(c.ops[0].H.dot, lambda v: multigrid.vcycle(c.ops, v), b, rtol=1e-13)[0])
    lam = np.asarray(krylov.pcg(c.ops[0].H.dot, lambda v: multigrid.vcycle(c.ops, v), p - pt, rtol=1e-13)[0])
    g_ref = adjoint.theta_gradient(c.ops[0], c.prm, c.ms[0], c.theta, p, lam)
    g = c.h.theta_grad(c.gpu(p), c.gpu(lam))
    assert rel_l2(c.host(g), g_ref[c.idx[0]]) < 1e-12


def test_autograd_against_oracle_and_finite_differences():
    c = case(2, 8, 2, theta_seed=gi.SEED_THETA)
    n = c.ops[0].ncells
    b = c.gpu(gi.rhs(n)).requires_grad_(True)
    th = c.gpu(c.theta).requires_grad_(True)
    kw = dict(rtol=1e-13, max_iter=400)
    p = hmg.HelmholtzSolve.apply(c.h, b, th, kw, kw)
    pt = c.gpu(gi.ptarget(n)) * p.detach().abs().max()
    loss = 0.5 * ((p - pt) ** 2).sum()
    loss.backward()
    # oracle gradients
    solve = lambda ops, rhs: krylov.pcg(ops[0].H.dot, lambda v: multigrid.vcycle(ops, v), rhs, rtol=1e-13,
                                        max_iter=400)[0]
    pt_or = c.oracle_order(c.host(pt))
    L_ref, lam_ref, g_ref, _ = adjoint.value_and_grad(c.ops, c.prm, c.ms[0], c.theta, gi.rhs(n), pt_or, solve)
    assert float(loss.detach()) == pytest.approx(L_ref, rel=1e-9)
    assert rel_l2(c.host(b.grad), lam_ref[c.idx[0]]) < 1e-9
    assert rel_l2(c.host(th.grad), g_ref[c.idx[0]]) < 1e-9
    # central differences on the GPU path (h = 1e-6), several directions
    with torch.no_grad():
        for v in gi.directions(n, 4):
            vg = c.gpu(v)
            Lp = 0.5 * ((hmg.HelmholtzSolve.apply(c.h, b, th + 1e-6 * vg, kw, kw) - pt) ** 2).sum()
            Lm = 0.5 * ((hmg.HelmholtzSolve.apply(c.h, b, th - 1e-6 * vg, kw, kw) - pt) ** 2).sum()
            fd = float(Lp - Lm) / 2e-6
            assert float((th.grad * vg).sum()) == pytest.approx(fd, rel=1e-5)


def test_tracing_counts_kernels_inside_graphs():
    """Tracing (CUDA events around selected kernels) also works when the
    iteration body runs as a CUDA graph; per V-cycle the finest level runs
    one sweep0, nu_pre - 1 + nu_post sweeps and one residual+restriction."""
    c = case(3, 16, 3)
    b = c.gpu(gi.rhs(c.ops[0].ncells))
    c.h.solve(b)                                   # captures the graph untraced
    c.h.profile_start(kernels=["sweep", "sweep0", "resid_restrict"], levels=[0])
    _, info = c.h.solve(b)
    rec = c.h.profile_stop()
    k = info["iterations"]
    assert rec[("sweep", 0)][0] == 3 * k
    assert rec[("sweep0", 0)][0] == k
    assert rec[("resid_restrict", 0)][0] == k
    assert all(ms > 0 for _, ms in rec.values())
    n0 = c.h.launch_count()
    c.h.solve(b)
    assert c.h.launch_count() > n0


def test_integer_pipe_conversions_match_hardware_bitwise():
    """FP64 -> FP32 (roundTiesToEven) and FP32 -> FP64 of the mixed cycle,
    against the hardware conversions, bit for bit: random values over the
    whole exponent range, exact ties, carries into the exponent, the float
    range limits, subnormals, zeros, infinities and NaN."""
    rng = np.random.default_rng(5)
    vals = [rng.standard_normal(200000) * np.exp(rng.uniform(-180, 180, 200000))]
    f = rng.standard_normal(5000).astype(np.float32).astype(np.float64)
    ulp = np.abs(f) * 2.0 ** -24
    vals += [f, f + ulp, f - ulp, f + 0.5 * ulp, f + 1.5 * ulp, f + 0.49 * ulp]      # ties and near-ties
    big = float(np.finfo(np.float32).max)
    vals.append(np.array([0.0, -0.0, 1.0, -1.0, big, -big, big * (1 + 2.0 ** -25), big * (1 + 2.0 ** -23),
                          2.0 ** -126, 2.0 ** -127, 2.0 ** -149, 2.0 ** -150, 1e-45, 1e-300, 1e300,
                          np.inf, -np.inf, np.nan, 1 - 2.0 ** -25, 1 + 2.0 ** -24, 1 + 3 * 2.0 ** -24]))
    x = torch.tensor(np.concatenate(vals), dtype=torch.float64, device=DEV)
    mine = hmg.convert(x, torch.float32)
    hw = x.to(torch.float32)
    assert torch.equal(mine.view(torch.int32), hw.view(torch.int32))
    back = hmg.convert(hw, torch.float64)
    assert torch.equal(back.view(torch.int64), hw.to(torch.float64).view(torch.int64))


def test_algorithmic_experiments_small():
    """The experiment drivers run and show what Sec. 6 reports: multigrid
    iteration counts that do not grow with resolution, and a single-level
    method that needs several times as many iterations."""
    from paper_1605_00492_gb300 import experiments
    g = experiments.grid_independence([3, 4], nlayers=16)
    assert all(row["true_rel_residual"] < 2e-8 for row in g)
    assert g[1]["iterations"] <= g[0]["iterations"] + 1
    c = experiments.cfl_sweep([8.0], refinement=3, nlayers=16, nlevels=3)
    assert c[0]["single_level"]["iterations"] > 2 * c[0]["multigrid"]["iterations"]
    hist = experiments.history(refinement=3, nlayers=16, nlevels=3)
    mg = hist["multigrid"]
    assert mg[-1] < 1e-8 and all(b < a for a, b in zip(mg, mg[1:]))


def test_caller_allocator_backs_the_context_and_solves_match_oracle():
    """hmg_build_hierarchy_with_allocator with the binding's torch_allocator:
    every device allocation of the context (levels, Krylov vectors, the CG
    loop state, the GMRES basis allocated on first use) comes from PyTorch's
    caching allocator, and the solves agree with the oracle as with the
    CUDA runtime's allocator (1e-9, iterations within 1)."""
    r, nz, L = 3, 16, 3
    ms = mesh.hierarchy(r, L)
    prm = helmholtz.Params(refinement=r, nlayers=nz)
    ops = helmholtz.assemble_hierarchy(ms, prm)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    h = hmg.Hierarchy(r, nz, L, allocator=hmg.torch_allocator())
    h.assemble()
    after_build = torch.cuda.memory_allocated()
    assert after_build > before
    cen, _ = h.export_mesh(0)
    idx = cell_permutation(column_permutation(cen, ms[0].centroid), nz)
    b = gi.rhs(ops[0].ncells)
    bg = torch.tensor(b[idx], dtype=torch.float64, device=DEV)
    V = lambda v: multigrid.vcycle(ops, v)
    refs = {"cg": krylov.pcg(ops[0].H.dot, V, b, rtol=1e-8),
            "gmres": krylov.fgmres(ops[0].H.dot, V, b, rtol=1e-8, restart=30)}
    used = []
    for krylov_name in ("cg", "gmres"):
        x_ref, info_ref = refs[krylov_name]
        x, info = h.solve(bg, krylov=krylov_name, rtol=1e-8, restart=30)
        assert info["converged"] == 1
        assert rel_l2(x.cpu().numpy(), x_ref[idx]) <= 1e-9
        assert abs(info["iterations"] - info_ref.iterations) <= 1
        del x
        torch.cuda.synchronize()
        used.append(torch.cuda.memory_allocated())
    assert used[1] > used[0] > after_build     # CG loop state, then the GMRES basis, from the same pool
    h.close()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() <= before + bg.numel() * 8
