"""Algorithmic experiments of Sec. 6 on synthetic shells, through the library.

    python -m paper_1605_00492_gb300.experiments [--quick]

Prints one JSON object with:

* ``grid``      iterations and solve time of the multigrid-preconditioned CG
                solve at fixed Courant number 8 for refinements 3..7 (64
                layers, levels down to refinement 2): the grid independence
                of Sec. 6 ("Algorithmic scaling");
* ``cfl``       iterations and solve times of the multigrid and the
                single-level method (two block-Jacobi vertical line
                relaxations, ``levels=1``) for Courant numbers 2..64 at
                81,920 x 64 cells (Fig. "Algorithmic scaling", left);
* ``history``   relative residual after each iteration for both methods at
                81,920 x 64 cells, Courant number 8 (the convergence history
                of Sec. 6);
* ``breakdown`` per-level, per-kernel device time of one multigrid solve
                (the per-level breakdown of Table "Multigrid breakdown");
* ``nlo``       next-to-lowest order on 5,120 x 64 cells (Table "GridSetup"):
                GMRES(30) iterations and solve time to 1e-5 with the
                multigrid (NLO level, p-coarsening, 4 lowest-order levels)
                and with the single-level method, for Courant numbers 2..32
                (Table "SingleNodePerformance" and Fig. "Algorithmic
                scaling", NLO rows), the same comparison for the NLO
                velocity-pressure system (7.9 million unknowns, the paper's NLO
                problem) and the per-kernel breakdown of one multigrid solve.

Right-hand sides are the seeded N(0,1) fields of ``hmg_inputs``; every
lowest-order solve runs to ||r|| / ||b|| < 1e-8 from x = 0, every NLO solve
to the paper's 1e-5.
"""
import argparse
import json

import torch

import hmg_inputs as gi

import paper_1605_00492_gb300 as hmg

DEV = "cuda:0"


def _solve(h, b, **kw):
    h.solve(b, raise_on_failure=False, **kw)          # warm-up (captures the graph)
    torch.cuda.synchronize()
    _, info = h.solve(b, raise_on_failure=False, **kw)
    return info


def grid_independence(refinements, nlayers=64):
    out = []
    for r in refinements:
        h = hmg.Hierarchy(r, nlayers, max(1, r - 1))   # coarsest level: refinement 2 throughout
        h.assemble()
        b = torch.tensor(gi.rhs(h.ncells), device=DEV)
        info = _solve(h, b)
        out.append({"refinement": r, "ncols": h.levels[0]["ncols"], "nlayers": nlayers, "nlevels": len(h.levels),
                    "iterations": info["iterations"], "solve_ms": round(info["solve_ms"], 3),
                    "true_rel_residual": info["true_rel_residual"]})
        h.close()
    return out


def cfl_sweep(cfls, refinement=6, nlayers=64, nlevels=5):
    h = hmg.Hierarchy(refinement, nlayers, nlevels)
    b = torch.tensor(gi.rhs(h.ncells), device=DEV)
    out = []
    for cfl in cfls:
        h.assemble(nu_cfl=cfl)
        row = {"nu_cfl": cfl}
        for name, levels in (("multigrid", 0), ("single_level", 1)):
            info = _solve(h, b, levels=levels, max_iter=2000)
            row[name] = {"iterations": info["iterations"], "solve_ms": round(info["solve_ms"], 3),
                         "converged": info["converged"]}
        out.append(row)
    h.close()
    return out


def history(refinement=6, nlayers=64, nlevels=5, cfl=8.0):
    """||r_k|| / ||b|| for k = 1, 2, ...: the k-th iterate of a solve from
    x = 0 is the same whether or not the solve stops there, so a solve capped
    at k iterations reports it."""
    h = hmg.Hierarchy(refinement, nlayers, nlevels)
    h.assemble(nu_cfl=cfl)
    b = torch.tensor(gi.rhs(h.ncells), device=DEV)
    out = {}
    for name, levels in (("multigrid", 0), ("single_level", 1)):
        full = _solve(h, b, levels=levels, max_iter=2000)
        res = []
        for k in range(1, full["iterations"] + 1):
            _, info = h.solve(b, levels=levels, max_iter=k, raise_on_failure=False)
            res.append(info["rel_residual"])
        out[name] = res
    h.close()
    return out


def breakdown(refinement=6, nlayers=64, nlevels=5):
    h = hmg.Hierarchy(refinement, nlayers, nlevels)
    h.assemble()
    b = torch.tensor(gi.rhs(h.ncells), device=DEV)
    out = {}
    for precision in ("fp64", "mixed"):
        h.solve(b, precision=precision)
        h.profile_start()
        _, info = h.solve(b, precision=precision)
        rec = h.profile_stop()
        out[precision] = {"iterations": info["iterations"],
                          "kernels": {f"{k}@{lev}": {"launches": n, "ms": round(ms, 4)}
                                      for (k, lev), (n, ms) in sorted(rec.items(), key=lambda kv: (kv[0][1], kv[0][0]))}}
    h.close()
    return out


def nlo(cfls=(2, 8, 32), refinement=4, nlayers=64, nlevels=4, precision="fp64"):
    h = hmg.Hierarchy(refinement, nlayers, nlevels)
    b = torch.tensor(gi.nlo_rhs(6 * gi.ncells(refinement, nlayers)), device=DEV)
    out = {"cfl": []}
    for cfl in cfls:
        h.assemble(nu_cfl=cfl)
        row = {"nu_cfl": cfl}
        for name, levels in (("multigrid", 0), ("single_level", 1)):
            kw = dict(rtol=1e-5, restart=30, levels=levels, max_iter=3000, precision=precision)
            h.nlo_solve(b, raise_on_failure=False, **kw)
            torch.cuda.synchronize()
            _, info = h.nlo_solve(b, raise_on_failure=False, **kw)
            row[name] = {"iterations": info["iterations"], "solve_ms": round(info["solve_ms"], 3),
                         "converged": info["converged"]}
        out["cfl"].append(row)
    # the velocity-pressure system (the paper's NLO problem, 7.9 M unknowns at
    # r4x64): GMRES(30) to 1e-5 with the Schur-complement preconditioner, H^^-1
    # by the multigrid or by the single-level method
    h.assemble()
    sizes = h.nlo_mixed_sizes()
    nu = sum(sizes) - sizes[3]
    R = torch.tensor(gi.mixed_rhs(nu, sizes[3]), device=DEV)
    Ru, Rp = R.clone(), R.clone()
    Ru[nu:] = 0
    Rp[:nu] = 0
    bvp = torch.cat([h.nlo_mixed_apply(Ru)[:nu], h.nlo_mixed_apply(Rp)[nu:]])
    out["velocity_pressure"] = {"unknowns": int(sum(sizes))}
    for name, levels in (("multigrid", 0), ("single_level", 1)):
        kw = dict(rtol=1e-5, restart=30, levels=levels, max_iter=3000, precision=precision)
        h.nlo_mixed_solve(bvp, raise_on_failure=False, **kw)
        torch.cuda.synchronize()
        _, info = h.nlo_mixed_solve(bvp, raise_on_failure=False, **kw)
        out["velocity_pressure"][name] = {"iterations": info["iterations"], "solve_ms": round(info["solve_ms"], 3),
                                          "converged": info["converged"]}
    h.nlo_solve(b, rtol=1e-5, precision=precision)
    h.profile_start()
    _, info = h.nlo_solve(b, rtol=1e-5, precision=precision)
    rec = h.profile_stop()
    out["breakdown"] = {"iterations": info["iterations"],
                        "kernels": {f"{k}@{lev}": {"launches": n, "ms": round(ms, 4)}
                                    for (k, lev), (n, ms) in sorted(rec.items(), key=lambda kv: (kv[0][1], kv[0][0]))}}
    h.close()
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--quick", action="store_true", help="smaller shells (refinement 5) and fewer Courant numbers")
    ap.add_argument("--only", choices=["grid", "cfl", "history", "breakdown", "nlo"], default=None,
                    help="run one experiment")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64",
                    help="form of the V-cycle in the NLO experiment")
    args = ap.parse_args()
    if not torch.cuda.is_available():
        raise SystemExit("a CUDA device is required")
    r = 5 if args.quick else 6
    runs = {
        "grid": lambda: grid_independence([3, 4, 5] if args.quick else [3, 4, 5, 6, 7]),
        "cfl": lambda: cfl_sweep([2, 8, 32] if args.quick else [2, 4, 8, 16, 32, 64], refinement=r),
        "history": lambda: history(refinement=r),
        "breakdown": lambda: breakdown(refinement=r),
        "nlo": lambda: nlo((8,) if args.quick else (2, 8, 32), precision=args.precision),
    }
    res = {k: f() for k, f in runs.items() if args.only in (None, k)}
    print(json.dumps(res))


if __name__ == "__main__":
    main()
