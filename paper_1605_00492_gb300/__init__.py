"""GB300 tensor-product multigrid solver for the lumped pressure-Helmholtz
operator of Mitchell & Mueller's LO (RT0 x DG0) discretisation on an
extruded icosahedral shell.

This module is argument marshalling only: every step of the path runs in the
CUDA kernels of ``libhmg.so`` (``include/hmg.h``).  PyTorch supplies device
memory and streams.  There is no CPU fallback: importing this package fails
if the library is missing.
"""
import ctypes
import os
from dataclasses import dataclass

import torch

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = _build.LIB

HMG_OK = 0
STATUS = {
    0: "HMG_OK", 1: "HMG_ERR_INVALID_ARG", 2: "HMG_ERR_CUDA", 3: "HMG_ERR_OOM",
    4: "HMG_ERR_NOT_CONVERGED", 5: "HMG_ERR_BREAKDOWN", 6: "HMG_ERR_NONFINITE", 7: "HMG_ERR_STATE",
}
FP64, FP32 = 0, 1
LAYOUT = {"column": 0, "tiled": 1}
PRECISION = {"fp64": 0, "mixed": 1}
KRYLOV = {"cg": 0, "fcg": 1, "gmres": 2}


class HMGError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class MeshParams(ctypes.Structure):
    _fields_ = [("refinement", ctypes.c_int), ("nlayers", ctypes.c_int), ("nlevels", ctypes.c_int),
                ("radius_m", ctypes.c_double), ("thickness_m", ctypes.c_double)]


class OpParams(ctypes.Structure):
    _fields_ = [("c", ctypes.c_double), ("N", ctypes.c_double), ("nu_cfl", ctypes.c_double),
                ("dx_m", ctypes.c_double), ("omega", ctypes.c_double)]


class SolveParams(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("krylov", ctypes.c_int), ("rtol", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("nu_pre", ctypes.c_int), ("nu_post", ctypes.c_int),
                ("n_coarse", ctypes.c_int), ("restart", ctypes.c_int), ("levels", ctypes.c_int),
                ("orth", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("true_rel_residual", ctypes.c_double), ("solve_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class KernelStat(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("level", ctypes.c_int), ("launches", ctypes.c_int),
                ("total_ms", ctypes.c_double)]


KERNELS = ["sweep0", "sweep", "prolong", "resid_restrict", "apply", "dot", "update_xr", "update_p", "layout",
           "resid_sq", "assembly", "theta_grad", "ortho", "nlo_sweep", "nlo_resid", "nlo_apply",
           "nlo_sweep0", "coarse_cycle", "halo"]


class PartInfo(ctypes.Structure):
    _fields_ = [("col_begin", ctypes.c_int32), ("col_end", ctypes.c_int32), ("ncols_padded", ctypes.c_int32),
                ("n_ghost", ctypes.c_int32), ("n_send", ctypes.c_int32)]


class LevelInfo(ctypes.Structure):
    _fields_ = [("refinement", ctypes.c_int), ("ncols", ctypes.c_int), ("ncols_padded", ctypes.c_int),
                ("nlayers", ctypes.c_int), ("ncells", ctypes.c_int64), ("ncells_padded", ctypes.c_int64)]


_P = ctypes.c_void_p
_I = ctypes.c_int
# hmg_alloc_fn / hmg_release_fn
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
RELEASE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
_SIGNATURES = {
    "hmg_build_hierarchy": [ctypes.POINTER(MeshParams), ctypes.POINTER(_P)],
    "hmg_build_hierarchy_with_allocator": [ctypes.POINTER(MeshParams), ALLOC_FN, RELEASE_FN, _P, ctypes.POINTER(_P)],
    "hmg_destroy": [_P],
    "hmg_get_level_info": [_P, _I, ctypes.POINTER(LevelInfo)],
    "hmg_export_mesh": [_P, _I, _P, _P],
    "hmg_assemble_helmholtz": [_P, ctypes.POINTER(OpParams), _P, _P],
    "hmg_apply": [_P, _I, _I, _I, _P, _P, _P],
    "hmg_apply_noalloc": [_P, _I, _P, _P, _P],
    "hmg_vcycle": [_P, _I, _I, _P, _P, _I, _I, _I, _P],
    "hmg_solve": [_P, _P, _P, ctypes.POINTER(SolveParams), ctypes.POINTER(SolveInfo), _P],
    "hmg_solve_host": [_P, _P, _P, ctypes.POINTER(SolveParams), ctypes.POINTER(SolveInfo), _P],
    "hmg_theta_grad": [_P, _P, _P, _P, _P],
    "hmg_mixed_sizes": [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                        ctypes.POINTER(ctypes.c_int64)],
    "hmg_export_edges": [_P, _P],
    "hmg_mixed_apply": [_P, _P, _P, _P, _P, _P],
    "hmg_mixed_solve": [_P, _P, _P, _P, _P, ctypes.POINTER(SolveParams), ctypes.POINTER(SolveInfo), _P],
    "hmg_nlo_size": [_P, ctypes.POINTER(ctypes.c_int64)],
    "hmg_export_vertices": [_P, _I, _P],
    "hmg_nlo_host_blocks": [ctypes.POINTER(MeshParams), ctypes.POINTER(OpParams), _P, _P, _P, _P, _P],
    "hmg_nlo_apply": [_P, _P, _P, _P],
    "hmg_nlo_vcycle": [_P, _I, _P, _P, _I, _I, _I, _I, _P],
    "hmg_nlo_solve": [_P, _P, _P, ctypes.POINTER(SolveParams), ctypes.POINTER(SolveInfo), _P],
    "hmg_nlo_mixed_sizes": [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                            ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)],
    "hmg_nlo_mixed_host_csr": [ctypes.POINTER(MeshParams), ctypes.POINTER(OpParams), ctypes.POINTER(ctypes.c_int64),
                               ctypes.POINTER(ctypes.c_int64), _P, _P, _P, _P],
    "hmg_nlo_mixed_apply": [_P, _P, _P, _P],
    "hmg_nlo_mixed_solve": [_P, _P, _P, ctypes.POINTER(SolveParams), ctypes.POINTER(SolveInfo), _P],
    "hmg_to_layout": [_P, _I, _I, _P, _I, _P, _P],
    "hmg_sync": [_P, _P],
    "hmg_convert_fp64_to_fp32": [_P, _P, ctypes.c_int64, _P],
    "hmg_convert_fp32_to_fp64": [_P, _P, ctypes.c_int64, _P],
    "hmg_set_coarse_fusion": [_P, _I],
    "hmg_measure_fp64_rate": [_P, ctypes.POINTER(ctypes.c_double), _P],
    "hmg_partition": [_P, _I],
    "hmg_partition_info": [_I, _I, _I, _I, _I, ctypes.POINTER(PartInfo)],
    "hmg_partition_tables": [_I, _I, _I, _I, _I, _P, _P, _P, _P, _P, _P],
    "hmg_profile_start": [_P, ctypes.c_uint, ctypes.c_uint],
    "hmg_profile_stop": [_P, ctypes.POINTER(KernelStat), _I, ctypes.POINTER(_I)],
    "hmg_launch_count": [_P, ctypes.POINTER(ctypes.c_int64)],
    "hmg_residual_history": [_P, _P, _I, ctypes.POINTER(_I)],
    "hmg_kernel_name": [_I],
    "hmg_last_error": [_P],
    "hmg_status_string": [_I],
}

_lib = None


def load_library(path=None):
    """Load libhmg.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1605_00492_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, args in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_char_p if name in ("hmg_last_error", "hmg_status_string", "hmg_kernel_name") \
            else ctypes.c_int
    if path == LIB_PATH:
        _lib = lib
    return lib


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


@dataclass
class Workload:
    refinement: int
    nlayers: int
    nlevels: int


class Allocator:
    """Device memory for a context from a caller's pair of callables:
    alloc(nbytes) -> device pointer as int (0 or None when out of memory),
    release(ptr).  The ctypes callbacks are kept alive with the object."""

    def __init__(self, alloc, release):
        def _alloc(nbytes, user):
            try:
                return alloc(int(nbytes)) or None
            except RuntimeError:          # the pool is exhausted
                return None

        def _release(ptr, user):
            release(ptr)
        self.alloc_fn = ALLOC_FN(_alloc)
        self.release_fn = RELEASE_FN(_release)


def torch_allocator(device=None):
    """An Allocator backed by PyTorch's CUDA caching allocator."""
    dev = torch.cuda.current_device() if device is None else device
    return Allocator(lambda n: torch.cuda.caching_allocator_alloc(n, dev), torch.cuda.caching_allocator_delete)


class Hierarchy:
    """Mesh hierarchy plus assembled operator on the current CUDA device.
    allocator: None (the CUDA runtime's cudaMalloc) or an Allocator, through
    which every device allocation of the context goes."""

    def __init__(self, refinement, nlayers, nlevels, radius_m=6.371e6, thickness_m=1.0e4, allocator=None):
        self.lib = load_library()
        self._ctx = _P()
        self._allocator = allocator
        p = MeshParams(refinement, nlayers, nlevels, radius_m, thickness_m)
        if allocator is None:
            st = self.lib.hmg_build_hierarchy(ctypes.byref(p), ctypes.byref(self._ctx))
        else:
            st = self.lib.hmg_build_hierarchy_with_allocator(ctypes.byref(p), allocator.alloc_fn,
                                                             allocator.release_fn, None, ctypes.byref(self._ctx))
        if st != HMG_OK:
            raise HMGError(st, self.lib.hmg_last_error(None).decode())
        self.refinement, self.nlayers, self.nlevels = refinement, nlayers, nlevels
        self.levels = [self.level_info(k) for k in range(nlevels)]
        self.ncells = self.levels[0]["ncells"]

    def _check(self, st, allow=()):
        if st != HMG_OK and st not in allow:
            raise HMGError(st, self.lib.hmg_last_error(self._ctx).decode())
        return st

    def close(self):
        if self._ctx:
            self.lib.hmg_destroy(self._ctx)
            self._ctx = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def level_info(self, level):
        info = LevelInfo()
        self._check(self.lib.hmg_get_level_info(self._ctx, level, ctypes.byref(info)))
        return {k: getattr(info, k) for k, _ in info._fields_}

    def export_mesh(self, level=0):
        import numpy as np
        nc = self.levels[level]["ncols"]
        cen = np.zeros((nc, 3), dtype=np.float64)
        nbr = np.zeros((nc, 3), dtype=np.int32)
        self._check(self.lib.hmg_export_mesh(self._ctx, level, cen.ctypes.data_as(_P), nbr.ctypes.data_as(_P)))
        return cen, nbr

    def assemble(self, theta=None, c=300.0, N=0.01, nu_cfl=8.0, dx_m=0.0, omega=0.8, stream=None):
        p = OpParams(c, N, nu_cfl, dx_m, omega)
        th = None
        if theta is not None:
            th = theta.contiguous()
            assert th.dtype == torch.float64 and th.is_cuda and th.numel() == self.ncells
        self._check(self.lib.hmg_assemble_helmholtz(self._ctx, ctypes.byref(p), _ptr(th) if th is not None else None,
                                                    _stream(stream)))
        return self

    def _len(self, level, layout):
        return self.levels[level]["ncells" if layout == "column" else "ncells_padded"]

    def apply(self, x, level=0, layout="column", out=None, stream=None):
        dtype = FP64 if x.dtype == torch.float64 else FP32
        assert x.is_cuda and x.numel() == self._len(level, layout)
        x = x.contiguous()
        y = out if out is not None else torch.empty_like(x)
        self._check(self.lib.hmg_apply(self._ctx, level, dtype, LAYOUT[layout], _ptr(x), _ptr(y), _stream(stream)))
        return y

    def apply_noalloc(self, x, level=0, out=None, stream=None):
        """y = H^ x (FP64, COLUMN layout) through hmg_apply_noalloc: no device
        memory is allocated by the library for the call (out must be given to
        avoid the allocation of the result tensor here)."""
        assert x.is_cuda and x.dtype == torch.float64 and x.numel() == self._len(level, "column")
        x = x.contiguous()
        y = out if out is not None else torch.empty_like(x)
        self._check(self.lib.hmg_apply_noalloc(self._ctx, level, _ptr(x), _ptr(y), _stream(stream)))
        return y

    def vcycle(self, r, precision="fp64", layout="column", nu_pre=2, nu_post=2, n_coarse=2, out=None, stream=None):
        assert r.is_cuda and r.dtype == torch.float64 and r.numel() == self._len(0, layout)
        r = r.contiguous()
        z = out if out is not None else torch.empty_like(r)
        self._check(self.lib.hmg_vcycle(self._ctx, PRECISION[precision], LAYOUT[layout], _ptr(r), _ptr(z),
                                        nu_pre, nu_post, n_coarse, _stream(stream)))
        return z

    def solve_params(self, precision="fp64", krylov="cg", rtol=1e-8, max_iter=500, nu_pre=2, nu_post=2,
                     n_coarse=2, restart=30, levels=0, orth=1):
        return SolveParams(PRECISION[precision], KRYLOV[krylov], rtol, max_iter, nu_pre, nu_post, n_coarse,
                           restart, levels, orth)

    def solve(self, b, out=None, stream=None, raise_on_failure=True, **kw):
        """x = H^^-1 b by V-cycle-preconditioned CG, flexible CG or GMRES(restart); returns (x, info dict)."""
        assert b.is_cuda and b.dtype == torch.float64 and b.numel() == self.ncells
        b = b.contiguous()
        x = out if out is not None else torch.empty_like(b)
        info = SolveInfo()
        p = self.solve_params(**kw)
        st = self.lib.hmg_solve(self._ctx, _ptr(b), _ptr(x), ctypes.byref(p), ctypes.byref(info), _stream(stream))
        d = info.as_dict()
        d["status"] = STATUS.get(st, st)
        if raise_on_failure:
            self._check(st)
        return x, d

    def solve_host(self, b_host, x_host, stream=None, raise_on_failure=True, **kw):
        """Solve with HOST tensors (pinned for asynchronous copies)."""
        assert not b_host.is_cuda and b_host.dtype == torch.float64 and b_host.numel() == self.ncells
        info = SolveInfo()
        p = self.solve_params(**kw)
        st = self.lib.hmg_solve_host(self._ctx, _ptr(b_host), _ptr(x_host), ctypes.byref(p), ctypes.byref(info),
                                     _stream(stream))
        d = info.as_dict()
        d["status"] = STATUS.get(st, st)
        if raise_on_failure:
            self._check(st)
        return x_host, d

    # ---- velocity-pressure system (Sec. 4.1) and its Schur-complement preconditioner (Sec. 4.2)

    def mixed_sizes(self):
        """(horizontal faces, vertical faces, cells) of the finest level."""
        h, v, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.hmg_mixed_sizes(self._ctx, ctypes.byref(h), ctypes.byref(v), ctypes.byref(c)))
        return h.value, v.value, c.value

    def export_edges(self):
        """(ne, 4) int32 array of (t, k, tn, kn) per edge."""
        import numpy as np
        nh, _, _ = self.mixed_sizes()
        ne = nh // self.levels[0]["nlayers"]
        e = np.zeros((ne, 4), dtype=np.int32)
        self._check(self.lib.hmg_export_edges(self._ctx, e.ctypes.data_as(_P)))
        return e

    def mixed_apply(self, u, p, stream=None):
        """(yu, yp) = A (u, p) for device FP64 tensors in the COLUMN layouts."""
        yu, yp = torch.empty_like(u), torch.empty_like(p)
        self._check(self.lib.hmg_mixed_apply(self._ctx, _ptr(u.contiguous()), _ptr(p.contiguous()), _ptr(yu), _ptr(yp),
                                             _stream(stream)))
        return yu, yp

    def mixed_solve(self, bu, bp, stream=None, raise_on_failure=True, **kw):
        """(u, p) = A^-1 (bu, bp) by GMRES(restart) with the Schur-complement
        preconditioner; keyword arguments as solve (rtol defaults to 1e-5 here,
        the paper's tolerance).  Returns (u, p, info dict)."""
        kw.setdefault("rtol", 1e-5)
        kw.setdefault("krylov", "gmres")
        u, p = torch.empty_like(bu), torch.empty_like(bp)
        info = SolveInfo()
        prm = self.solve_params(**kw)
        st = self.lib.hmg_mixed_solve(self._ctx, _ptr(bu.contiguous()), _ptr(bp.contiguous()), _ptr(u), _ptr(p),
                                      ctypes.byref(prm), ctypes.byref(info), _stream(stream))
        d = info.as_dict()
        d["status"] = STATUS.get(st, st)
        if raise_on_failure:
            self._check(st)
        return u, p, d

    # ---- next-to-lowest order (Table "FiniteElements": DG1 pressure, BDFM1 x DG1 velocity)

    def nlo_size(self):
        """Length of an NLO vector: 6 unknowns per cell of the finest level."""
        n = ctypes.c_int64()
        self._check(self.lib.hmg_nlo_size(self._ctx, ctypes.byref(n)))
        return n.value

    def export_vertices(self, level=0):
        """(ncols, 3, 3) unit-sphere vertices of each column's triangle, in
        the order that numbers the NLO unknowns."""
        import numpy as np
        v = np.zeros((self.levels[level]["ncols"], 3, 3))
        self._check(self.lib.hmg_export_vertices(self._ctx, level, v.ctypes.data_as(_P)))
        return v

    def nlo_apply(self, x, out=None, stream=None):
        """y = H^ x for the NLO operator (COLUMN layout, FP64 device tensors)."""
        y = out if out is not None else torch.empty_like(x)
        self._check(self.lib.hmg_nlo_apply(self._ctx, _ptr(x.contiguous()), _ptr(y), _stream(stream)))
        return y

    def nlo_vcycle(self, r, precision="fp64", nu_pre=2, nu_post=2, n_coarse=2, levels=0, out=None, stream=None):
        """z = V r: one NLO V-cycle (p-coarsening to the lowest-order hierarchy)."""
        z = out if out is not None else torch.empty_like(r)
        self._check(self.lib.hmg_nlo_vcycle(self._ctx, PRECISION[precision], _ptr(r.contiguous()), _ptr(z), nu_pre,
                                            nu_post, n_coarse, levels, _stream(stream)))
        return z

    def nlo_solve(self, b, out=None, stream=None, raise_on_failure=True, **kw):
        """x = H^^-1 b for the NLO operator by GMRES(restart) with the NLO
        V-cycle; keyword arguments as solve.  Returns (x, info dict)."""
        kw.setdefault("krylov", "gmres")
        x = out if out is not None else torch.empty_like(b)
        info = SolveInfo()
        prm = self.solve_params(**kw)
        st = self.lib.hmg_nlo_solve(self._ctx, _ptr(b.contiguous()), _ptr(x), ctypes.byref(prm), ctypes.byref(info),
                                    _stream(stream))
        d = info.as_dict()
        d["status"] = STATUS.get(st, st)
        if raise_on_failure:
            self._check(st)
        return x, d

    # ---- next-to-lowest-order velocity-pressure system

    def nlo_mixed_sizes(self):
        """(horizontal edge, horizontal interior, vertical, pressure) block lengths."""
        v = [ctypes.c_int64() for _ in range(4)]
        self._check(self.lib.hmg_nlo_mixed_sizes(self._ctx, *(ctypes.byref(x) for x in v)))
        return tuple(x.value for x in v)

    def nlo_mixed_apply(self, x, out=None, stream=None):
        """y = A x, NLO mixed COLUMN layout, FP64 device tensors."""
        y = out if out is not None else torch.empty_like(x)
        self._check(self.lib.hmg_nlo_mixed_apply(self._ctx, _ptr(x.contiguous()), _ptr(y), _stream(stream)))
        return y

    def nlo_mixed_solve(self, b, out=None, stream=None, raise_on_failure=True, **kw):
        """x = A^-1 b by GMRES(restart) with the Schur-complement preconditioner
        and the NLO V-cycle; keyword arguments as solve (rtol defaults to the
        paper's 1e-5).  Returns (x, info dict)."""
        kw.setdefault("rtol", 1e-5)
        kw.setdefault("krylov", "gmres")
        x = out if out is not None else torch.empty_like(b)
        info = SolveInfo()
        prm = self.solve_params(**kw)
        st = self.lib.hmg_nlo_mixed_solve(self._ctx, _ptr(b.contiguous()), _ptr(x), ctypes.byref(prm),
                                          ctypes.byref(info), _stream(stream))
        d = info.as_dict()
        d["status"] = STATUS.get(st, st)
        if raise_on_failure:
            self._check(st)
        return x, d

    def theta_grad(self, p, lam, out=None, stream=None):
        g = out if out is not None else torch.empty_like(p)
        self._check(self.lib.hmg_theta_grad(self._ctx, _ptr(p.contiguous()), _ptr(lam.contiguous()), _ptr(g),
                                            _stream(stream)))
        return g

    def to_layout(self, v, src="column", dst="tiled", level=0, stream=None):
        out = torch.zeros(self._len(level, dst), dtype=torch.float64, device=v.device)
        self._check(self.lib.hmg_to_layout(self._ctx, level, LAYOUT[src], _ptr(v.contiguous()), LAYOUT[dst],
                                           _ptr(out), _stream(stream)))
        return out

    def measure_fp64_rate(self, stream=None):
        """FP64 FMA throughput of this device in TFLOP/s (include/hmg.h)."""
        v = ctypes.c_double()
        self._check(self.lib.hmg_measure_fp64_rate(self._ctx, ctypes.byref(v), _stream(stream)))
        return v.value

    def partition(self, nparts):
        """Run as nparts parts of the horizontal domain decomposition, emulated
        on this device (include/hmg.h, hmg_partition); 1 = unpartitioned."""
        self._check(self.lib.hmg_partition(self._ctx, int(nparts)))

    def set_coarse_fusion(self, enable):
        """Run the coarse end of each V-cycle as one cooperative kernel (True)
        or as one kernel per pass (False, the default); same results."""
        self._check(self.lib.hmg_set_coarse_fusion(self._ctx, 1 if enable else 0))

    def profile_start(self, kernels=None, levels=None):
        """Bracket launches of the named kernel classes on the given levels with
        CUDA events (all when None)."""
        kmask = 0xFFFFFFFF if kernels is None else sum(1 << KERNELS.index(k) for k in kernels)
        lmask = 0xFFFFFFFF if levels is None else sum(1 << int(l) for l in levels)
        self._check(self.lib.hmg_profile_start(self._ctx, kmask, lmask))

    def profile_stop(self):
        """Records {(kernel, level): (launches, total_ms)} since profile_start."""
        cap = 512
        buf = (KernelStat * cap)()
        n = _I()
        self._check(self.lib.hmg_profile_stop(self._ctx, buf, cap, ctypes.byref(n)))
        return {(KERNELS[buf[i].kernel], buf[i].level): (buf[i].launches, buf[i].total_ms)
                for i in range(min(n.value, cap))}

    def residual_history(self):
        """Relative residual after each iteration of the last solve (numpy array)."""
        import numpy as np
        n = _I()
        self._check(self.lib.hmg_residual_history(self._ctx, None, 0, ctypes.byref(n)))
        out = np.zeros(n.value)
        if n.value:
            self._check(self.lib.hmg_residual_history(self._ctx, out.ctypes.data_as(_P), n.value, ctypes.byref(n)))
        return out

    def launch_count(self):
        n = ctypes.c_int64()
        self._check(self.lib.hmg_launch_count(self._ctx, ctypes.byref(n)))
        return n.value

    def sync(self, stream=None):
        self._check(self.lib.hmg_sync(self._ctx, _stream(stream)))


def partition_tables(refinement, nlevels, nparts, part, level):
    """Host-only (no GPU): the horizontal domain decomposition of the column
    hierarchy for one part and one partitioned level (include/hmg.h,
    hmg_partition_tables).  Returns a dict: col_begin, col_end, ncols_padded
    and the int32 arrays ghost_col, ghost_owner, ghost_owner_local, local_nbr
    (n_own, 3), send_col, send_to."""
    import numpy as np
    lib = load_library()
    info = PartInfo()
    st = lib.hmg_partition_info(refinement, nlevels, nparts, part, level, ctypes.byref(info))
    if st != 0:
        raise HMGError(st, lib.hmg_last_error(None).decode())
    n_own = info.col_end - info.col_begin
    out = dict(col_begin=info.col_begin, col_end=info.col_end, ncols_padded=info.ncols_padded,
               ghost_col=np.zeros(info.n_ghost, np.int32), ghost_owner=np.zeros(info.n_ghost, np.int32),
               ghost_owner_local=np.zeros(info.n_ghost, np.int32), local_nbr=np.zeros((n_own, 3), np.int32),
               send_col=np.zeros(info.n_send, np.int32), send_to=np.zeros(info.n_send, np.int32))
    st = lib.hmg_partition_tables(refinement, nlevels, nparts, part, level,
                                  *(out[k].ctypes.data_as(_P) for k in ("ghost_col", "ghost_owner",
                                                                         "ghost_owner_local", "local_nbr",
                                                                         "send_col", "send_to")))
    if st != 0:
        raise HMGError(st, lib.hmg_last_error(None).decode())
    return out


def nlo_host_blocks(refinement, nlayers, c=300.0, N=0.01, nu_cfl=8.0, dx_m=0.0, omega=0.8, radius_m=6.371e6,
                    thickness_m=1.0e4):
    """Host-only assembly of the NLO operator's blocks on the finest mesh
    (no GPU): returns dict(diag (ncols, nlayers, 6, 6), sub (same), nbr_blocks
    (ncols, 3, 6, 6), nbr (ncols, 3), verts (ncols, 3, 3))."""
    import numpy as np
    lib = load_library()
    nc = 20 * 4 ** refinement
    mp = MeshParams(refinement, nlayers, 1, radius_m, thickness_m)
    op = OpParams(c, N, nu_cfl, dx_m, omega)
    out = dict(diag=np.zeros((nc, nlayers, 6, 6)), sub=np.zeros((nc, nlayers, 6, 6)),
               nbr_blocks=np.zeros((nc, 3, 6, 6)), nbr=np.zeros((nc, 3), dtype=np.int32), verts=np.zeros((nc, 3, 3)))
    st = lib.hmg_nlo_host_blocks(ctypes.byref(mp), ctypes.byref(op), *(out[k].ctypes.data_as(_P) for k in
                                                                        ("diag", "sub", "nbr_blocks", "nbr", "verts")))
    if st != 0:
        raise HMGError(st, lib.hmg_last_error(None).decode())
    return out


def nlo_mixed_host_csr(refinement, nlayers, c=300.0, N=0.01, nu_cfl=8.0, dx_m=0.0, omega=0.8, radius_m=6.371e6,
                       thickness_m=1.0e4):
    """Host-only assembly of the NLO velocity-pressure matrix (no GPU):
    returns (scipy CSR matrix A, edge list (ne, 4) int32)."""
    import numpy as np
    import scipy.sparse as sp
    lib = load_library()
    mp = MeshParams(refinement, nlayers, 1, radius_m, thickness_m)
    op = OpParams(c, N, nu_cfl, dx_m, omega)
    n, nnz = ctypes.c_int64(), ctypes.c_int64()
    st = lib.hmg_nlo_mixed_host_csr(ctypes.byref(mp), ctypes.byref(op), ctypes.byref(n), ctypes.byref(nnz),
                                    None, None, None, None)
    if st != 0:
        raise HMGError(st, lib.hmg_last_error(None).decode())
    ptr = np.zeros(n.value + 1, dtype=np.int64)
    col = np.zeros(nnz.value, dtype=np.int32)
    val = np.zeros(nnz.value)
    edges = np.zeros((30 * 4 ** refinement, 4), dtype=np.int32)
    st = lib.hmg_nlo_mixed_host_csr(ctypes.byref(mp), ctypes.byref(op), ctypes.byref(n), ctypes.byref(nnz),
                                    ptr.ctypes.data_as(_P), col.ctypes.data_as(_P), val.ctypes.data_as(_P),
                                    edges.ctypes.data_as(_P))
    if st != 0:
        raise HMGError(st, lib.hmg_last_error(None).decode())
    return sp.csr_matrix((val, col, ptr), shape=(n.value, n.value)), edges


def convert(x, dtype, stream=None):
    """FP64 <-> FP32 on the GPU with the library's integer-pipe conversion."""
    lib = load_library()
    assert x.is_cuda and x.is_contiguous()
    out = torch.empty(x.shape, dtype=dtype, device=x.device)
    if x.dtype == torch.float64 and dtype == torch.float32:
        st = lib.hmg_convert_fp64_to_fp32(_ptr(x), _ptr(out), x.numel(), _stream(stream))
    elif x.dtype == torch.float32 and dtype == torch.float64:
        st = lib.hmg_convert_fp32_to_fp64(_ptr(x), _ptr(out), x.numel(), _stream(stream))
    else:
        raise ValueError("convert: FP64 -> FP32 or FP32 -> FP64 only")
    if st != HMG_OK:
        raise HMGError(st, "conversion failed")
    return out


from .autograd import HelmholtzSolve  # noqa: E402  (needs Hierarchy)

__all__ = ["Hierarchy", "HelmholtzSolve", "HMGError", "load_library", "LIB_PATH"]
