"""Thin ctypes binding of libalstokes.so (include/alstokes.h).

Argument marshalling only: every step of the solver runs in the CUDA
library.  Device vectors are passed as torch CUDA tensors (their data
pointers); setup/solve arrays may be NumPy arrays or torch tensors.  There is
no CPU fallback: importing works anywhere, but every call needs the built
library and a CUDA device, and fails loudly otherwise.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, Structure, byref, c_double, c_int, c_longlong, c_void_p

import numpy as np

from . import build as _build

ALS_OK, ALS_EINVAL, ALS_ENOMEM, ALS_ECUDA, ALS_ENOTSPD, ALS_ENOTCONV, ALS_EBREAKDOWN, ALS_ETIMEOUT = range(8)
STATUS_NAMES = ["ALS_OK", "ALS_EINVAL", "ALS_ENOMEM", "ALS_ECUDA", "ALS_ENOTSPD", "ALS_ENOTCONV",
                "ALS_EBREAKDOWN", "ALS_ETIMEOUT"]
ALS_COEFF_SCALAR, ALS_COEFF_TENSOR = 0, 1
ALS_PREC_FP64, ALS_PREC_FP32 = 0, 1
ALS_MODE_FP64, ALS_MODE_MIXED = 0, 1
ALS_BATCH_MERGED, ALS_BATCH_BRANCHES = 0, 1
ALS_SMOOTH_GMRES, ALS_SMOOTH_RICHARDSON = 0, 1
ALS_TRANSFER_ROBUST, ALS_TRANSFER_STANDARD = 0, 1
ALS_SCHUR_P1, ALS_SCHUR_P2 = 0, 1
ALS_CYCLE_V, ALS_CYCLE_F = 0, 1
ALS_FACT_FULL, ALS_FACT_UPPER, ALS_FACT_LOWER, ALS_FACT_DIAG = 0, 1, 2, 3
ALS_SETUP_AUTO, ALS_SETUP_FP64 = 0, 1
ALS_STORE_FP32, ALS_STORE_BF16 = 0, 1
ALS_STATIC_SCRATCH_BYTES = 32 * 1024 * 1024


class als_mesh(Structure):
    _fields_ = [("dim", c_int), ("n", c_int * 3), ("levels", c_int)]


class als_coeff(Structure):
    _fields_ = [("kind", c_int), ("qp", POINTER(c_void_p)), ("mu_eff", POINTER(c_void_p))]


class als_options(Structure):
    _fields_ = [("smoother", c_int), ("sweeps", c_int), ("tau", c_double), ("transfer", c_int),
                ("schur", c_int), ("mode", c_int), ("rtol", c_double), ("maxit", c_int),
                ("cycle", c_int), ("fact", c_int), ("setup", c_int), ("order", c_int), ("store", c_int)]


class als_newton_params(Structure):
    _fields_ = [("mu_ref", c_double), ("tau_y", c_double), ("rtol", c_double), ("maxit", c_int),
                ("max_halvings", c_int)]


class als_newton_info(Structure):
    _fields_ = [("iterations", c_int), ("linear_iterations", c_int), ("converged", c_int), ("res0", c_double),
                ("res_final", c_double)]


class als_solve_info(Structure):
    _fields_ = [("iterations", c_int), ("vcycles", c_int), ("converged", c_int), ("res0", c_double),
                ("res_final", c_double), ("solve_ms", c_double)]


# name -> (restype, argtypes); the exported C ABI
SIGNATURES = {
    "als_default_options": (None, [POINTER(als_options)]),
    "als_create": (c_int, [POINTER(als_mesh), POINTER(als_coeff), c_double, POINTER(als_options), c_void_p,
                           POINTER(c_void_p)]),
    "als_destroy": (c_int, [c_void_p]),
    "als_apply_agamma": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p]),
    "als_vcycle": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    "als_star_smooth": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p]),
    "als_prolong": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p]),
    "als_restrict": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p]),
    "als_coarse_solve": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    "als_apply_stokes": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "als_patch_inverse": (c_int, [c_void_p, c_int, c_longlong, c_void_p]),
    "als_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, POINTER(als_solve_info)]),
    "als_last_error": (ctypes.c_char_p, [c_void_p]),
    "als_update_coefficients": (c_int, [c_void_p, POINTER(als_coeff)]),
    "als_profile": (c_int, [c_void_p, c_int]),
    "als_profile_read": (c_int, [c_void_p, POINTER(c_double), POINTER(c_longlong)]),
    "als_profile_read_kernel": (c_int, [c_void_p, c_int, POINTER(c_double), POINTER(c_longlong)]),
    "als_kernel_launches": (c_longlong, []),
    "als_star_smooth_static": (c_int, [c_int, POINTER(c_int), c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "als_measure_fma_peaks": (c_int, [POINTER(c_double), POINTER(c_double), c_void_p]),
    "als_batch_create": (c_int, [c_int, POINTER(als_mesh), POINTER(als_coeff), POINTER(c_double),
                                 POINTER(als_options), c_void_p, POINTER(c_void_p)]),
    "als_batch_destroy": (c_int, [c_void_p]),
    "als_batch_context": (c_int, [c_void_p, c_int, POINTER(c_void_p)]),
    "als_batch_solve": (c_int, [c_void_p, POINTER(c_void_p), POINTER(c_void_p), POINTER(c_void_p),
                                POINTER(c_void_p), POINTER(c_void_p), POINTER(als_solve_info)]),
    "als_batch_vcycle": (c_int, [c_void_p, c_int, POINTER(c_void_p), POINTER(c_void_p)]),
    "als_batch_last_error": (ctypes.c_char_p, [c_void_p]),
    "als_batch_set_mode": (c_int, [c_void_p, c_int]),
    "als_batch_get_mode": (c_int, [c_void_p, POINTER(c_int)]),
    "als_batch_merged_plan": (c_int, [c_void_p, POINTER(c_int), POINTER(c_int), POINTER(ctypes.c_float),
                                      POINTER(ctypes.c_longlong)]),
    "als_batch_set_grouping": (c_int, [c_void_p, c_int]),
    "als_batch_merged_tune": (c_int, [c_void_p, c_int, c_int, POINTER(c_int), POINTER(c_int),
                                      POINTER(ctypes.c_float), POINTER(c_int)]),
    "als_autotune_info": (c_int, [c_void_p, c_int, POINTER(c_int), POINTER(ctypes.c_float)]),
    "als_set_patch_kernel": (c_int, [c_void_p, c_int, c_int]),
    "als_load_patch_inverses": (c_int, [c_void_p, c_int, c_void_p]),
    "als_load_coarse_inverse": (c_int, [c_void_p, c_void_p]),
    "als_set_wait_limit": (c_int, [c_void_p, c_int]),
    "als_solve_history": (c_int, [c_void_p, POINTER(c_double), c_int, POINTER(c_int)]),
    "als_newton_default_params": (None, [POINTER(als_newton_params)]),
    "als_newton_solve": (c_int, [c_void_p, POINTER(als_newton_params), c_void_p, c_void_p, c_void_p, c_void_p,
                                 POINTER(als_newton_info)]),
    "als_newton_history": (c_int, [c_void_p, POINTER(c_double), POINTER(c_int), c_int, POINTER(c_int)]),
}

_LIB = None


class ALSError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")


def library_path():
    return _build.LIB


def load(build_if_missing=False):
    """Load libalstokes.so (building it first if asked).  Raises if it is absent."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA extension {path} is not built; run paper_2107_00820_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _ptr(a):
    """Data pointer of a torch tensor or a NumPy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("arrays must be contiguous")
        return c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return c_void_p(a.ctypes.data)
    raise TypeError(f"unsupported array type {type(a)}")


def _check_dtype(a, prec):
    if a is None:
        return
    name = str(a.dtype)
    want = "float64" if prec == ALS_PREC_FP64 else "float32"
    if not name.endswith(want):
        raise TypeError(f"expected {want} data for prec={prec}, got {name}")


def _check_f64_len(a, need, what):
    """An FP64 array (NumPy or torch, host or device) of at least `need` entries."""
    if a is None:
        raise ValueError(f"{what}: an array is required")
    name = str(a.dtype)
    if not name.endswith("float64"):
        raise TypeError(f"{what}: expected float64 data, got {name}")
    size = int(a.numel()) if hasattr(a, "numel") else int(a.size)
    if size < need:
        raise ValueError(f"{what}: {size} entries, the context needs {need}")


def _cuda_tensor(a):
    if not (hasattr(a, "is_cuda") and a.is_cuda):
        raise TypeError("this entry point takes CUDA tensors (device pointers)")


def default_options(**kw):
    lib = load()
    o = als_options()
    lib.als_default_options(byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def pressure_per_cell(dim, order):
    """Pressure unknowns per cell, dim P_(order-1)^disc = C(order - 1 + dim, dim)."""
    import math
    return math.comb(order - 1 + dim, dim)


class Context:
    """An als_ctx: setup once (als_create), then apply / V-cycle / solve."""

    def __init__(self, dim, n, levels, coeffs, gamma, mu_eff=None, stream=None, **options):
        lib = load()
        n = (n,) * dim if np.isscalar(n) else tuple(n)
        self.dim, self.n, self.levels, self.gamma = dim, n, levels, float(gamma)
        mesh = als_mesh(dim, (c_int * 3)(*(list(n) + [1] * (3 - len(n)))), levels)
        kind = ALS_COEFF_TENSOR if mu_eff is not None else ALS_COEFF_SCALAR
        self._keep = [np.ascontiguousarray(c, dtype=np.float64) if isinstance(c, np.ndarray) else c for c in coeffs]
        qp = (c_void_p * levels)(*[_ptr(c) for c in self._keep])
        mu = None
        if mu_eff is not None:
            self._keep_mu = [np.ascontiguousarray(c, dtype=np.float64) if isinstance(c, np.ndarray) else c
                             for c in mu_eff]
            mu = (c_void_p * levels)(*[_ptr(c) for c in self._keep_mu])
        coeff = als_coeff(kind, qp, mu)
        self._kind = kind
        self.options = default_options(**options)
        out = c_void_p()
        st = lib.als_create(byref(mesh), byref(coeff), self.gamma, byref(self.options),
                            c_void_p(stream) if stream else None, byref(out))
        if st != ALS_OK:
            raise ALSError(st, "als_create: " + lib.als_last_error(None).decode())
        self._ctx = out
        self._lib = lib

    # sizes -----------------------------------------------------------------
    def level_n(self, level):
        f = 2 ** (self.levels - 1 - level)
        return tuple(v // f for v in self.n)

    @property
    def order(self):
        return int(getattr(self, "options", None).order) if getattr(self, "options", None) is not None else 2

    def nu(self, level=None):
        nl = self.level_n(self.levels - 1 if level is None else level)
        return self.dim * int(np.prod([self.order * v + 1 for v in nl]))

    def npres(self):
        return pressure_per_cell(self.dim, self.order) * int(np.prod(self.n))

    # calls -----------------------------------------------------------------
    def _call(self, name, *args):
        st = getattr(self._lib, name)(self._ctx, *args)
        if st != ALS_OK:
            raise ALSError(st, self._lib.als_last_error(self._ctx).decode())
        return st

    def apply_agamma(self, x, y, level=None, prec=ALS_PREC_FP64):
        level = self.levels - 1 if level is None else level
        _cuda_tensor(x); _cuda_tensor(y); _check_dtype(x, prec); _check_dtype(y, prec)
        self._call("als_apply_agamma", level, prec, _ptr(x), _ptr(y))

    def vcycle(self, b, x, prec=ALS_PREC_FP64):
        _cuda_tensor(b); _cuda_tensor(x); _check_dtype(b, prec); _check_dtype(x, prec)
        self._call("als_vcycle", prec, _ptr(b), _ptr(x))

    def star_smooth(self, level, r, z, prec=ALS_PREC_FP64):
        _cuda_tensor(r); _cuda_tensor(z); _check_dtype(r, prec)
        self._call("als_star_smooth", level, prec, _ptr(r), _ptr(z))

    def prolong(self, level, xc, xf, prec=ALS_PREC_FP64):
        _cuda_tensor(xc); _cuda_tensor(xf); _check_dtype(xc, prec)
        self._call("als_prolong", level, prec, _ptr(xc), _ptr(xf))

    def restrict(self, level, rf, rc, prec=ALS_PREC_FP64):
        _cuda_tensor(rf); _cuda_tensor(rc); _check_dtype(rf, prec)
        self._call("als_restrict", level, prec, _ptr(rf), _ptr(rc))

    def coarse_solve(self, b, x, prec=ALS_PREC_FP64):
        _cuda_tensor(b); _cuda_tensor(x); _check_dtype(b, prec)
        self._call("als_coarse_solve", prec, _ptr(b), _ptr(x))

    def apply_stokes(self, u, p, yu, yp):
        for a in (u, p, yu, yp):
            _cuda_tensor(a); _check_dtype(a, ALS_PREC_FP64)
        self._call("als_apply_stokes", _ptr(u), _ptr(p), _ptr(yu), _ptr(yp))

    def patch_inverse(self, level, vertex):
        np_ = self.patch_dofs()
        out = np.zeros((np_, np_))
        self._call("als_patch_inverse", level, int(vertex), _ptr(out))
        return out

    def solve(self, f_qp, u_bc=None, r2=None, u=None, p=None, check=True):
        """Returns (u, p, info); inputs/outputs may be host (NumPy) or device (torch)."""
        if u is None:
            u = np.zeros(self.nu())
        if p is None:
            p = np.zeros(self.npres())
        info = als_solve_info()
        st = self._lib.als_solve(self._ctx, _ptr(f_qp), _ptr(u_bc), _ptr(r2), _ptr(u), _ptr(p), byref(info))
        if st != ALS_OK and (check or st != ALS_ENOTCONV):
            raise ALSError(st, self._lib.als_last_error(self._ctx).decode())
        return u, p, info

    def update_coefficients(self, coeffs, mu_eff=None):
        """Re-run the setup for new per-level coefficients (host or device arrays)."""
        keep = [np.ascontiguousarray(c, dtype=np.float64) if isinstance(c, np.ndarray) else c for c in coeffs]
        qp = (c_void_p * self.levels)(*[_ptr(c) for c in keep])
        mu = None
        if mu_eff is not None:
            keep_mu = [np.ascontiguousarray(c, dtype=np.float64) if isinstance(c, np.ndarray) else c for c in mu_eff]
            mu = (c_void_p * self.levels)(*[_ptr(c) for c in keep_mu])
        coeff = als_coeff(self._kind, qp, mu)
        self._call("als_update_coefficients", byref(coeff))

    def profile(self, on=True):
        self._call("als_profile", 1 if on else 0)

    def profile_read(self):
        ms, n = c_double(), c_longlong()
        self._call("als_profile_read", byref(ms), byref(n))
        return ms.value, n.value

    def autotune_info(self, level):
        """(chosen FP32 patch-kernel variant, [ms per launch of variants 0, 1, 2]) of a level."""
        v = c_int()
        ms = (ctypes.c_float * 3)()
        self._call("als_autotune_info", c_int(level), byref(v), ms)
        return v.value, list(ms)

    def set_patch_kernel(self, level, variant):
        self._call("als_set_patch_kernel", c_int(level), c_int(variant))

    def patch_dofs(self):
        """Dofs of an interior vertex star: d (2k - 1)^d."""
        return self.dim * (2 * self.order - 1) ** self.dim

    def coarse_free_dofs(self):
        """Free velocity dofs of the coarsest level: d prod(k n_0 - 1)."""
        return self.dim * int(np.prod([self.order * v - 1 for v in self.level_n(0)]))

    def load_patch_inverses(self, level, packed):
        """Replace the patch inverses of `level` by FP64 ones packed by diagonals
        (nverts x stride, host or device); the FP32 copies are rounded from them.
        The array's dtype and length are checked here, so that the library's copy
        never reads past the caller's buffer."""
        if not 1 <= int(level) < self.levels:
            raise ValueError(f"level must be in [1, {self.levels})")
        np_ = self.patch_dofs()
        stride = (np_ * (np_ + 1) // 2 + 3) // 4 * 4
        nverts = int(np.prod([v + 1 for v in self.level_n(level)]))
        _check_f64_len(packed, nverts * stride, "packed patch inverses")
        self._call("als_load_patch_inverses", c_int(level), _ptr(packed))

    def load_coarse_inverse(self, inv):
        """Replace the coarse inverse (nfree x nfree FP64, host or device); dtype and
        length checked as for load_patch_inverses."""
        nf = self.coarse_free_dofs()
        _check_f64_len(inv, nf * nf, "coarse inverse")
        self._call("als_load_coarse_inverse", _ptr(inv))

    def set_wait_limit(self, polls):
        """Test switch: poll limit of the FP32 smoother kernel's waits (< 0: default)."""
        self._call("als_set_wait_limit", c_int(polls))

    def solve_history(self):
        """Residual history of the last solve: |b|, then the estimate after each iteration."""
        cnt = c_int()
        self._call("als_solve_history", None, 0, byref(cnt))
        out = (c_double * max(cnt.value, 1))()
        self._call("als_solve_history", out, cnt.value, byref(cnt))
        return np.array(out[: cnt.value])

    def newton_solve(self, f_qp, u_bc=None, u=None, p=None, check=True, **params):
        """Newton's method for the viscoplastic rheology (als_newton_solve); params are the
        fields of als_newton_params (mu_ref, tau_y, rtol, maxit, max_halvings).  Returns
        (u, p, info); inputs/outputs may be host (NumPy) or device (torch) arrays."""
        prm = als_newton_params()
        self._lib.als_newton_default_params(byref(prm))
        for k, v in params.items():
            if not hasattr(prm, k):
                raise KeyError(k)
            setattr(prm, k, v)
        u = np.zeros(self.nu()) if u is None else u
        p = np.zeros(self.npres()) if p is None else p
        info = als_newton_info()
        st = self._lib.als_newton_solve(self._ctx, byref(prm), _ptr(f_qp), _ptr(u_bc), _ptr(u), _ptr(p), byref(info))
        if st != ALS_OK and (check or st != ALS_ENOTCONV):
            raise ALSError(st, self._lib.als_last_error(self._ctx).decode())
        return u, p, info

    def newton_history(self):
        """(residual norms, FGMRES iterations per step) of the last Newton solve."""
        cnt = c_int()
        self._call("als_newton_history", None, None, 0, byref(cnt))
        res = (c_double * max(cnt.value, 1))()
        its = (c_int * max(cnt.value, 1))()
        self._call("als_newton_history", res, its, cnt.value, byref(cnt))
        return np.array(res[: cnt.value]), list(its[: cnt.value])

    def profile_read_kernel(self, kind):
        """(total ms, launches) of kernel class `kind` (0 patch kernel, 1 operator apply)."""
        ms, n = c_double(), c_longlong()
        self._call("als_profile_read_kernel", c_int(kind), byref(ms), byref(n))
        return ms.value, n.value

    def close(self):
        if getattr(self, "_ctx", None) is not None:
            self._lib.als_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# module-level functions with the C names (thin pass-through)
class Batch:
    """An als_batch: independent instances solved together.

    instances: list of dicts with keys dim, n, levels, coeffs (per-level arrays),
    gamma and optionally mu_eff and options (keyword options of default_options).
    """

    def __init__(self, instances, stream=None):
        lib = load()
        k = len(instances)
        meshes = (als_mesh * k)()
        coeffs = (als_coeff * k)()
        gammas = (c_double * k)()
        opts = (als_options * k)()
        self._keep = []
        self.shapes = []
        self._meta = []
        for i, ins in enumerate(instances):
            dim, levels = ins["dim"], ins["levels"]
            n = (ins["n"],) * dim if np.isscalar(ins["n"]) else tuple(ins["n"])
            meshes[i] = als_mesh(dim, (c_int * 3)(*(list(n) + [1] * (3 - len(n)))), levels)
            keep = [np.ascontiguousarray(c, dtype=np.float64) if isinstance(c, np.ndarray) else c
                    for c in ins["coeffs"]]
            qp = (c_void_p * levels)(*[_ptr(c) for c in keep])
            mu = None
            if ins.get("mu_eff") is not None:
                keep_mu = [np.ascontiguousarray(c, dtype=np.float64) if isinstance(c, np.ndarray) else c
                           for c in ins["mu_eff"]]
                mu = (c_void_p * levels)(*[_ptr(c) for c in keep_mu])
                keep += keep_mu
            coeffs[i] = als_coeff(ALS_COEFF_TENSOR if mu is not None else ALS_COEFF_SCALAR, qp, mu)
            self._keep += [keep, qp, mu]
            gammas[i] = float(ins["gamma"])
            opts[i] = default_options(**ins.get("options", {}))
            order = int(opts[i].order)
            nu = dim * int(np.prod([order * v + 1 for v in n]))
            self.shapes.append((nu, pressure_per_cell(dim, order) * int(np.prod(n))))
            self._meta.append((dim, n, levels, opts[i]))
        out = c_void_p()
        st = lib.als_batch_create(k, meshes, coeffs, gammas, opts, c_void_p(stream) if stream else None, byref(out))
        if st != ALS_OK:
            raise ALSError(st, "als_batch_create: " + lib.als_last_error(None).decode())
        self._b = out
        self._lib = lib
        self.count = k

    def _check(self, st):
        if st != ALS_OK:
            raise ALSError(st, self._lib.als_batch_last_error(self._b).decode())

    def solve(self, f_qp, u_bc=None, r2=None, u=None, p=None, check=True):
        """Solves every instance; returns (u list, p list, info list)."""
        k = self.count
        u = u if u is not None else [np.zeros(s[0]) for s in self.shapes]
        p = p if p is not None else [np.zeros(s[1]) for s in self.shapes]
        arr = lambda xs: (c_void_p * k)(*[_ptr(x) for x in xs]) if xs is not None else None  # noqa: E731
        infos = (als_solve_info * k)()
        st = self._lib.als_batch_solve(self._b, arr(f_qp), arr(u_bc), arr(r2), arr(u), arr(p), infos)
        if st != ALS_OK and (check or st != ALS_ENOTCONV):
            self._check(st)
        return u, p, list(infos)

    def vcycle(self, b, x, prec=ALS_PREC_FP64):
        for t in list(b) + list(x):
            _cuda_tensor(t); _check_dtype(t, prec)
        k = self.count
        self._check(self._lib.als_batch_vcycle(self._b, prec, (c_void_p * k)(*[_ptr(t) for t in b]),
                                               (c_void_p * k)(*[_ptr(t) for t in x])))

    @property
    def mode(self):
        """ALS_BATCH_MERGED or ALS_BATCH_BRANCHES (the execution form of the FP32 cycles)."""
        m = c_int()
        self._check(self._lib.als_batch_get_mode(self._b, byref(m)))
        return m.value

    def set_mode(self, mode):
        self._check(self._lib.als_batch_set_mode(self._b, int(mode)))

    def merged_plan(self):
        """(grouping, groups, ms per grouping [5], kernels of one merged cycle of the batch)."""
        g, n, kern = c_int(), c_int(), ctypes.c_longlong()
        ms = (ctypes.c_float * 5)()
        self._check(self._lib.als_batch_merged_plan(self._b, byref(g), byref(n), ms, byref(kern)))
        return g.value, n.value, list(ms), kern.value

    def set_grouping(self, grouping):
        """Fix the merged cycles' grouping (0 .. 4), or -1 to let the tuner choose."""
        self._check(self._lib.als_batch_set_grouping(self._b, int(grouping)))

    def merged_tune(self, group, level):
        """(products variant, interior variant, ms[6], batch indices of the group's instances)."""
        pv, iv = c_int(), c_int()
        ms = (ctypes.c_float * 6)()
        idx = (c_int * self.count)(*([-1] * self.count))
        self._check(self._lib.als_batch_merged_tune(self._b, int(group), int(level), byref(pv), byref(iv), ms, idx))
        return pv.value, iv.value, list(ms), [i for i in idx if i >= 0]

    def instance(self, i):
        """Instance i as a Context (owned by the batch: closing it does nothing)."""
        ptr = c_void_p()
        self._check(self._lib.als_batch_context(self._b, c_int(i), byref(ptr)))
        ctx = Context.__new__(_BorrowedContext)
        ctx._ctx, ctx._lib = ptr, self._lib
        dim, n, levels, options = self._meta[i]
        ctx.dim, ctx.n, ctx.levels, ctx.options = dim, n, levels, options
        return ctx

    def close(self):
        if getattr(self, "_b", None) is not None:
            self._lib.als_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


class _BorrowedContext(Context):
    """A context owned by a batch."""

    def close(self):
        self._ctx = None


def als_create(dim, n, levels, coeffs, gamma, **kw):
    return Context(dim, n, levels, coeffs, gamma, **kw)


def als_destroy(ctx):
    ctx.close()


def als_apply_agamma(ctx, level, prec, x, y):
    ctx.apply_agamma(x, y, level, prec)


def als_vcycle(ctx, prec, b, x):
    ctx.vcycle(b, x, prec)


def als_solve(ctx, f_qp, u_bc, r2, u, p):
    return ctx.solve(f_qp, u_bc, r2, u, p)


def als_kernel_launches():
    return int(load().als_kernel_launches())


def als_star_smooth_static(dim, n, prec, inv, r, z, stream=None):
    """Allocation-free smoother (scratch in a fixed device array); queued on `stream`.

    inv, r and z must be CUDA tensors of the precision's dtype holding at least
    (n+1)^d packed inverses and d (2n+1)^d vector entries (checked here, so that no host
    pointer or short buffer reaches the kernels)."""
    for a in (inv, r, z):
        _cuda_tensor(a)
        _check_dtype(a, prec)
    if dim in (2, 3) and len(n) >= dim and all(1 <= int(v) <= 4096 for v in n[:dim]):
        np_ = dim * 3 ** dim
        stride = ((np_ * (np_ + 1) // 2) + 3) & ~3
        nverts = int(np.prod([int(v) + 1 for v in n[:dim]]))
        nu = dim * int(np.prod([2 * int(v) + 1 for v in n[:dim]]))
        elt = 8 if prec == ALS_PREC_FP64 else 4
        if nverts * np_ * elt > ALS_STATIC_SCRATCH_BYTES:
            pass                    # beyond the fixed scratch: the library refuses it (ALS_EINVAL)
        elif inv.numel() < nverts * stride:
            raise ValueError(f"inv holds {inv.numel()} entries, the mesh needs {nverts * stride}")
        elif r.numel() < nu or z.numel() < nu:
            raise ValueError(f"r and z need {nu} entries")
    n = (list(n) + [1, 1, 1])[:3]
    st = load().als_star_smooth_static(dim, (c_int * 3)(*n), prec, _ptr(inv), _ptr(r), _ptr(z),
                                       c_void_p(stream) if stream else None)
    if st != ALS_OK:
        raise ALSError(st, "als_star_smooth_static failed")


def als_measure_fma_peaks(stream=None):
    """Measured (FP32, FP64) FMA throughput of the current GPU in TFLOP/s."""
    f32, f64 = c_double(), c_double()
    st = load().als_measure_fma_peaks(byref(f32), byref(f64), c_void_p(stream) if stream else None)
    if st != ALS_OK:
        raise ALSError(st, "als_measure_fma_peaks failed")
    return f32.value, f64.value
