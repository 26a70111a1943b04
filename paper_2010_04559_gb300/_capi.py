"""ctypes binding of libamgt.so (include/amgt.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Device buffers are passed as torch CUDA tensors (their
data_ptr); host arrays as NumPy arrays.  Importing this module loads the
library and raises if it is missing -- there is no fallback.
"""
import ctypes
import os

import numpy as np

from . import build as _build

AMGT_OK = 0
AMGT_ERR_ARG = -1
AMGT_ERR_CUDA = -2
AMGT_ERR_NOMEM = -3
AMGT_ERR_NOT_CONVERGED = -4
AMGT_ERR_BREAKDOWN = -5
AMGT_ERR_NAN = -6
AMGT_ERR_DEVICE_TIMEOUT = -7
AMGT_ERR_STATE = -8
AMGT_ERR_UNSUPPORTED = -9

AMGT_F64 = 0
AMGT_F32 = 1
AMGT_F32_BF16TC = 2
AMGT_F64_SPLIT = 3
AMGT_F32_TC3 = 4

AMGT_PREC_NONE = 0
AMGT_PREC_SWEEP = 1
AMGT_PREC_MG = 2
AMGT_MODE_F64 = 0
AMGT_MODE_MIXED = 1

AMGT_MAX_HIST = 1024

AMGT_TUNE_GS_KERNEL = 1
AMGT_TUNE_SWEEP_GROUP = 2
AMGT_TUNE_SWEEP_STAGES = 3
AMGT_TUNE_GS_GRID_BLOCKS = 4
AMGT_TUNE_GS_CLUSTER = 5
AMGT_TUNE_KERNEL_TIMERS = 6
AMGT_TUNE_GRAPHS = 7
AMGT_TUNE_FP64_SCATTER = 8
AMGT_TUNE_SPLIT_ROWS = 9
AMGT_TUNE_SWEEP_KERNEL = 10
AMGT_TUNE_F32_SCATTER = 11
AMGT_TUNE_TEST_SWEEP_HOLD = 12
AMGT_TUNE_COARSE_F64 = 13
AMGT_TUNE_GS_FORM = 14
AMGT_KRYLOV_GMRES, AMGT_KRYLOV_BICGSTAB = 0, 1
AMGT_KT_SWEEP, AMGT_KT_APPLY_L, AMGT_KT_SCATTER_PREP, AMGT_KT_SCATTER_TC = 0, 1, 2, 3
AMGT_KT_SCATTER_F32, AMGT_KT_COARSE_GS, AMGT_KT_SCATTER_F64 = 4, 5, 6
AMGT_KT_SPLIT_TC, AMGT_KT_SPLIT_AUX = 7, 8
AMGT_KT_TC3, AMGT_KT_TC3_PREP = 9, 10
AMGT_KT_COUNT = 11

# every exported symbol of include/amgt.h
EXPORTS = [
    "amgt_create", "amgt_destroy", "amgt_last_error", "amgt_set_stream", "amgt_sync",
    "amgt_query_launches", "amgt_query_kernel_time", "amgt_query_kernel_stats",
    "amgt_set_mesh_cartesian", "amgt_set_materials", "amgt_set_angular_uniform",
    "amgt_set_angular_aniso", "amgt_set_multigrid", "amgt_set_source_iso",
    "amgt_set_boundary", "amgt_set_tuning", "amgt_query_sizes", "amgt_solve", "amgt_op_source",
    "amgt_op_sweep", "amgt_op_apply_L", "amgt_op_scatter", "amgt_op_apply_A",
    "amgt_op_restrict", "amgt_op_prolong", "amgt_op_smooth", "amgt_op_coarse_gs",
    "amgt_op_coarse_gs_noalloc",
    "amgt_op_vcycle", "amgt_op_scalar_flux",
    "amgt_set_adjoint", "amgt_response", "amgt_response_gradients",
    "amgt_autotune", "amgt_solve_batch", "amgt_setup_batch",
]


class amgt_options(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart", ctypes.c_int), ("maxit", ctypes.c_int),
                ("precond", ctypes.c_int), ("mode", ctypes.c_int),
                ("device_ptrs", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("inner_maxit", ctypes.c_int), ("krylov", ctypes.c_int)]


class amgt_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("outer_iterations", ctypes.c_int),
                ("relres", ctypes.c_double), ("seconds", ctypes.c_double),
                ("nhist", ctypes.c_int), ("hist", ctypes.c_double * AMGT_MAX_HIST)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_PD = ctypes.POINTER(ctypes.c_double)
_PI64 = ctypes.POINTER(ctypes.c_int64)
_PI = ctypes.POINTER(ctypes.c_int)

_SIGS = {
    "amgt_create": ([ctypes.POINTER(_P), _I, _P], _I),
    "amgt_destroy": ([_P], None),
    "amgt_last_error": ([_P], ctypes.c_char_p),
    "amgt_set_stream": ([_P, _P], _I),
    "amgt_sync": ([_P], _I),
    "amgt_query_launches": ([_PI64], _I),
    "amgt_query_kernel_time": ([_P, _I, _I, _PD, _PI64], _I),
    "amgt_query_kernel_stats": ([_P, _I, _I, _PD, _PI64, _PD], _I),
    "amgt_set_mesh_cartesian": ([_P, _I, _PI64, _PD, _PD], _I),
    "amgt_set_materials": ([_P, _PD, _PD, ctypes.POINTER(ctypes.c_int32), _I, _I, _PD], _I),
    "amgt_set_angular_uniform": ([_P, _I, _I], _I),
    "amgt_set_angular_aniso": ([_P, _I, _PD, _I], _I),
    "amgt_set_multigrid": ([_P, _I, _PI, _I, _I, _I], _I),
    "amgt_set_source_iso": ([_P, _PD], _I),
    "amgt_set_boundary": ([_P, _I, _I, _PD], _I),
    "amgt_set_tuning": ([_P, _I, _I], _I),
    "amgt_query_sizes": ([_P, _I, _PI64, _PI64], _I),
    "amgt_solve": ([_P, ctypes.POINTER(amgt_options), _P, _P, _P,
                    ctypes.POINTER(amgt_stats)], _I),
    "amgt_op_source": ([_P, _I, _I, _P], _I),
    "amgt_op_sweep": ([_P, _I, _I, _P, _P], _I),
    "amgt_op_apply_L": ([_P, _I, _I, _P, _P], _I),
    "amgt_op_scatter": ([_P, _I, _I, _P, _P], _I),
    "amgt_op_apply_A": ([_P, _I, _I, _P, _P], _I),
    "amgt_op_restrict": ([_P, _I, _I, _P, _P], _I),
    "amgt_op_prolong": ([_P, _I, _I, _P, _P], _I),
    "amgt_op_smooth": ([_P, _I, _I, _I, _P, _P], _I),
    "amgt_op_coarse_gs": ([_P, _I, _I, _P, _P], _I),
    "amgt_op_coarse_gs_noalloc": ([_P, _I, _I, _P, _P], _I),
    "amgt_op_vcycle": ([_P, _I, _P, _P], _I),
    "amgt_op_scalar_flux": ([_P, _I, _I, _P, _P], _I),
    "amgt_set_adjoint": ([_P, _I], _I),
    "amgt_response": ([_P, _I, _P, _PD], _I),
    "amgt_response_gradients": ([_P, _I, _P, _P, _P, _P, _P], _I),
    "amgt_autotune": ([_P, _I, _PI], _I),
    "amgt_solve_batch": ([ctypes.POINTER(_P), _I, ctypes.POINTER(amgt_options),
                          ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(amgt_stats), _I],
                         _I),
    "amgt_setup_batch": ([ctypes.POINTER(_P), _I, _I], _I),
}


def load(path=None):
    """Load the built library (never builds implicitly unless asked)."""
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError("libamgt.so is not built: run __graft_entry__.build() "
                           "or python -m paper_2010_04559_gb300.build")
    lib = ctypes.CDLL(path)
    for name, (args, res) in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load()
    return _lib


def amgt_query_launches():
    """Kernels launched by the library in this process so far."""
    n = ctypes.c_int64()
    rc = lib().amgt_query_launches(ctypes.byref(n))
    if rc != AMGT_OK:
        raise AmgtError(rc, "amgt_query_launches failed")
    return n.value


class AmgtError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"amgt error {code}: {msg}")
        self.code = code


def _dptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _np(a, dtype):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


class Context:
    """Owns one amgt_ctx; methods are one-to-one with the C entry points."""

    def __init__(self, device=0, stream=None):
        self.lib = lib()
        h = ctypes.c_void_p()
        s = ctypes.c_void_p(stream) if stream else ctypes.c_void_p()
        rc = self.lib.amgt_create(ctypes.byref(h), int(device), s)
        if rc != AMGT_OK:
            raise AmgtError(rc, "amgt_create failed (is a CUDA device visible?)")
        self.h = h

    def close(self):
        if self.h:
            self.lib.amgt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, allow=()):
        if rc != AMGT_OK and rc not in allow:
            raise AmgtError(rc, self.lib.amgt_last_error(self.h).decode())
        return rc

    # ---- problem statement
    def amgt_set_stream(self, stream):
        return self._check(self.lib.amgt_set_stream(self.h, ctypes.c_void_p(stream)))

    def amgt_sync(self):
        return self._check(self.lib.amgt_sync(self.h))

    def amgt_set_mesh_cartesian(self, dim, ncell, lo, hi):
        nc = _np(list(ncell) + [1] * (3 - len(ncell)), np.int64)
        lo = _np(list(lo)[:3] + [0.0] * (3 - len(lo)), np.float64)
        hi = _np(list(hi)[:3] + [1.0] * (3 - len(hi)), np.float64)
        return self._check(self.lib.amgt_set_mesh_cartesian(
            self.h, int(dim), nc.ctypes.data_as(_PI64), lo.ctypes.data_as(_PD),
            hi.ctypes.data_as(_PD)))

    def amgt_set_materials(self, sigma_t, sigma_s, N, fmom, mat_id=None):
        """fmom: f[N+1] (one shape) or f[nmat][N+1] with mat_id[C]."""
        st = _np(sigma_t, np.float64)
        ss = _np(sigma_s, np.float64)
        fm = _np(np.atleast_2d(np.asarray(fmom, dtype=np.float64)), np.float64)
        nmat = fm.shape[0]
        mid = None if mat_id is None else _np(mat_id, np.int32)
        pm = (ctypes.POINTER(ctypes.c_int32)() if mid is None
              else mid.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        return self._check(self.lib.amgt_set_materials(
            self.h, st.ctypes.data_as(_PD), ss.ctypes.data_as(_PD), pm, int(nmat), int(N),
            fm.ctypes.data_as(_PD)))

    def amgt_set_angular_uniform(self, basis, level):
        return self._check(self.lib.amgt_set_angular_uniform(self.h, int(basis), int(level)))

    def amgt_set_angular_aniso(self, basis, axis, lmax):
        ax = _np(axis, np.float64)
        return self._check(self.lib.amgt_set_angular_aniso(
            self.h, int(basis), ax.ctypes.data_as(_PD), int(lmax)))

    def amgt_set_multigrid(self, nlevels, Nr, nu_pre, nu_post, coarse_sweeps):
        nr = _np(Nr, np.int32)
        return self._check(self.lib.amgt_set_multigrid(
            self.h, int(nlevels), nr.ctypes.data_as(_PI), int(nu_pre), int(nu_post),
            int(coarse_sweeps)))

    def amgt_set_source_iso(self, q):
        qq = _np(q, np.float64)
        return self._check(self.lib.amgt_set_source_iso(self.h, qq.ctypes.data_as(_PD)))

    def amgt_set_boundary(self, face, kind, value=0.0):
        """value: a number (kinds 0-2), or for kind 3 the eight numbers
        (S, Omega_b[3], u0, u1, v0, v1)."""
        p = _np(np.atleast_1d(np.asarray(value, dtype=np.float64)).ravel(), np.float64)
        return self._check(self.lib.amgt_set_boundary(self.h, int(face), int(kind),
                                                      p.ctypes.data_as(_PD)))

    def amgt_set_tuning(self, key, value):
        return self._check(self.lib.amgt_set_tuning(self.h, int(key), int(value)))

    def amgt_query_kernel_time(self, kernel, reset=False):
        """(milliseconds, launches) timed for one AMGT_KT_* kernel class."""
        ms = ctypes.c_double(0.0)
        n = ctypes.c_int64(0)
        self._check(self.lib.amgt_query_kernel_time(self.h, int(kernel), 1 if reset else 0,
                                                    ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def amgt_query_kernel_stats(self, kernel, reset=False):
        """(milliseconds, launches, algorithmic work in bytes or flop) timed
        for one AMGT_KT_* kernel class."""
        ms = ctypes.c_double(0.0)
        n = ctypes.c_int64(0)
        w = ctypes.c_double(0.0)
        self._check(self.lib.amgt_query_kernel_stats(self.h, int(kernel), 1 if reset else 0,
                                                     ctypes.byref(ms), ctypes.byref(n),
                                                     ctypes.byref(w)))
        return ms.value, n.value, w.value

    def amgt_query_sizes(self, level=0):
        a = ctypes.c_int64()
        b = ctypes.c_int64()
        self._check(self.lib.amgt_query_sizes(self.h, int(level), ctypes.byref(a),
                                              ctypes.byref(b)))
        return a.value, b.value

    def amgt_solve(self, tol=1e-8, restart=20, maxit=1000, precond=AMGT_PREC_MG,
                   mode=AMGT_MODE_F64, x0=None, psi=None, phi=None, device_ptrs=False,
                   inner_tol=0.0, inner_maxit=200, allow_not_converged=False,
                   krylov=0):
        """Host mode: x0/psi/phi are NumPy float64 arrays (psi/phi allocated when
        None).  Device mode: torch CUDA float64 tensors.  krylov: 0 GMRES,
        1 BiCGStab."""
        opt = amgt_options(float(tol), int(restart), int(maxit), int(precond), int(mode),
                           1 if device_ptrs else 0, float(inner_tol), int(inner_maxit),
                           int(krylov))
        st = amgt_stats()
        nsdof, nadof = self.amgt_query_sizes(0)
        if device_ptrs:
            px, pp, pf = _dptr(x0), _dptr(psi), _dptr(phi)
        else:
            if psi is None:
                psi = np.empty((nsdof, nadof))
            if phi is None:
                phi = np.empty(nsdof)
            assert psi.dtype == np.float64 and psi.flags.c_contiguous
            assert phi.dtype == np.float64 and phi.flags.c_contiguous
            px = ctypes.c_void_p(0 if x0 is None else _np(x0, np.float64).ctypes.data)
            pp = ctypes.c_void_p(psi.ctypes.data)
            pf = ctypes.c_void_p(phi.ctypes.data)
        allow = (AMGT_ERR_NOT_CONVERGED,) if allow_not_converged else ()
        rc = self._check(self.lib.amgt_solve(self.h, ctypes.byref(opt), px, pp, pf,
                                             ctypes.byref(st)), allow)
        return psi, phi, st, rc

    # ---- operators on torch CUDA tensors
    @staticmethod
    def _dtype_code(t, tc=False):
        """tc: False (plain), True (BF16 tensor cores for FP32, split form for
        FP64) or "tc3" (FP32: the FP16 three-product tensor-core form)."""
        import torch
        if t.dtype == torch.float64:
            return AMGT_F64_SPLIT if tc else AMGT_F64
        if t.dtype == torch.float32:
            if tc == "tc3":
                return AMGT_F32_TC3
            return AMGT_F32_BF16TC if tc else AMGT_F32
        raise TypeError("buffers must be float64 or float32 CUDA tensors")

    @staticmethod
    def _req(*ts):
        for t in ts:
            if not (t.is_cuda and t.is_contiguous()):
                raise ValueError("operator buffers must be contiguous CUDA tensors")

    def amgt_op_source(self, level, f):
        self._req(f)
        return self._check(self.lib.amgt_op_source(self.h, level, self._dtype_code(f), _dptr(f)))

    def amgt_op_sweep(self, level, b, psi):
        self._req(b, psi)
        return self._check(self.lib.amgt_op_sweep(self.h, level, self._dtype_code(b),
                                                  _dptr(b), _dptr(psi)))

    def amgt_op_apply_L(self, level, x, y, tc=False):
        """tc=True with float64 buffers: double-float arithmetic (AMGT_F64_SPLIT)."""
        self._req(x, y)
        return self._check(self.lib.amgt_op_apply_L(self.h, level, self._dtype_code(x, tc),
                                                    _dptr(x), _dptr(y)))

    def amgt_op_scatter(self, level, x, y, tc=False):
        self._req(x, y)
        return self._check(self.lib.amgt_op_scatter(self.h, level, self._dtype_code(x, tc),
                                                    _dptr(x), _dptr(y)))

    def amgt_op_apply_A(self, level, x, y, tc=False):
        self._req(x, y)
        return self._check(self.lib.amgt_op_apply_A(self.h, level, self._dtype_code(x, tc),
                                                    _dptr(x), _dptr(y)))

    def amgt_op_restrict(self, level, rf, rc):
        self._req(rf, rc)
        return self._check(self.lib.amgt_op_restrict(self.h, level, self._dtype_code(rf),
                                                     _dptr(rf), _dptr(rc)))

    def amgt_op_prolong(self, level, xc, xf):
        self._req(xc, xf)
        return self._check(self.lib.amgt_op_prolong(self.h, level, self._dtype_code(xc),
                                                    _dptr(xc), _dptr(xf)))

    def amgt_op_smooth(self, level, nu, f, phi, tc=False):
        self._req(f, phi)
        return self._check(self.lib.amgt_op_smooth(self.h, level, self._dtype_code(f, tc), nu,
                                                   _dptr(f), _dptr(phi)))

    def amgt_op_coarse_gs(self, sweeps, f, phi):
        self._req(f, phi)
        return self._check(self.lib.amgt_op_coarse_gs(self.h, self._dtype_code(f), sweeps,
                                                      _dptr(f), _dptr(phi)))

    def amgt_op_coarse_gs_noalloc(self, sweeps, f, phi):
        """Coarse Gauss-Seidel without any device allocation (fixed scratch)."""
        self._req(f, phi)
        return self._check(self.lib.amgt_op_coarse_gs_noalloc(
            self.h, self._dtype_code(f), sweeps, _dptr(f), _dptr(phi)))

    def amgt_op_vcycle(self, f, phi, tc=False):
        self._req(f, phi)
        return self._check(self.lib.amgt_op_vcycle(self.h, self._dtype_code(f, tc), _dptr(f),
                                                   _dptr(phi)))

    def amgt_op_scalar_flux(self, level, psi, phi):
        self._req(psi, phi)
        return self._check(self.lib.amgt_op_scalar_flux(self.h, level, self._dtype_code(psi),
                                                        _dptr(psi), _dptr(phi)))

    def amgt_autotune(self, what=3):
        """(patches per block, copy stages, Gauss-Seidel kernel, cached)."""
        ch = (ctypes.c_int * 4)()
        self._check(self.lib.amgt_autotune(self.h, int(what), ch))
        return tuple(ch)

    # ---- adjoint and gradients
    def amgt_set_adjoint(self, on):
        return self._check(self.lib.amgt_set_adjoint(self.h, 1 if on else 0))

    @staticmethod
    def _mem(x):
        """(device flag, pointer) of a torch CUDA float64 tensor or a NumPy
        float64 array."""
        if isinstance(x, np.ndarray):
            assert x.dtype == np.float64 and x.flags.c_contiguous
            return 0, ctypes.c_void_p(x.ctypes.data)
        assert x.dtype.__str__() == "torch.float64" and x.is_contiguous()
        return 1, _dptr(x)

    def amgt_response(self, psi):
        dev, p = self._mem(psi)
        R = ctypes.c_double(0.0)
        self._check(self.lib.amgt_response(self.h, dev, p, ctypes.byref(R)))
        return R.value

    def amgt_response_gradients(self, psi, lam, dsigt, dsigs, dfmom):
        """Fill dsigt [C], dsigs [C], dfmom [N+1] or [nmat][N+1] (same memory
        space as psi)."""
        dev, p = self._mem(psi)
        dev2, l = self._mem(lam)
        assert dev == dev2
        outs = [self._mem(a) for a in (dsigt, dsigs, dfmom)]
        assert all(o[0] == dev for o in outs)
        return self._check(self.lib.amgt_response_gradients(self.h, dev, p, l, outs[0][1],
                                                            outs[1][1], outs[2][1]))


def amgt_solve_batch(contexts, psis, phis=None, tol=1e-8, restart=20, maxit=1000,
                     precond=AMGT_PREC_MG, mode=AMGT_MODE_MIXED, inner_tol=0.0,
                     inner_maxit=200, nthreads=0, allow_not_converged=False):
    """Solve the problems of `contexts` concurrently (one stream each) into the
    torch CUDA float64 tensors `psis` (and `phis`); returns the stats list."""
    n = len(contexts)
    opt = amgt_options(float(tol), int(restart), int(maxit), int(precond), int(mode), 1,
                       float(inner_tol), int(inner_maxit), 0)
    hs = (_P * n)(*[c.h for c in contexts])
    pp = (_P * n)(*[_dptr(p).value for p in psis])
    pf = (_P * n)(*[_dptr(p).value for p in phis]) if phis is not None else None
    st = (amgt_stats * n)()
    rc = lib().amgt_solve_batch(hs, n, ctypes.byref(opt), pp, pf, st, int(nthreads))
    allow = (AMGT_ERR_NOT_CONVERGED,) if allow_not_converged else ()
    if rc != AMGT_OK and rc not in allow:
        raise AmgtError(rc, "amgt_solve_batch failed: " +
                        "; ".join(c.lib.amgt_last_error(c.h).decode() for c in contexts[:3]))
    return list(st)


def amgt_setup_batch(contexts, nthreads=0):
    """Build the set-up tables of `contexts` concurrently (host threads, one
    stream per context), instead of at each context's first use."""
    n = len(contexts)
    hs = (_P * n)(*[c.h for c in contexts])
    rc = lib().amgt_setup_batch(hs, n, int(nthreads))
    if rc != AMGT_OK:
        raise AmgtError(rc, "amgt_setup_batch failed: " +
                        "; ".join(c.lib.amgt_last_error(c.h).decode() for c in contexts[:3]))


def context_from_problem(prob, device=0, stream=None, aniso=None):
    """Create a context and pass a workloads-style problem dict through the
    set_* entry points (marshalling only)."""
    ctx = Context(device, stream)
    dim = prob["dim"]
    ctx.amgt_set_mesh_cartesian(dim, prob["ncell"], prob["lo"], prob["hi"])
    ctx.amgt_set_materials(prob["sigma_t"], prob["sigma_s"], prob["N"], prob["fmom"],
                           prob.get("mat_id"))
    basis = 1 if prob["basis"] == "lin" else 0
    if aniso is None:
        ctx.amgt_set_angular_uniform(basis, prob["level"])
    else:
        axis, lmax = aniso
        ctx.amgt_set_angular_aniso(basis, axis, lmax)
    mg = prob.get("mg")
    if mg:
        ctx.amgt_set_multigrid(mg["nlevels"], mg["Nr"], mg["nu_pre"], mg["nu_post"],
                               mg["coarse_sweeps"])
    ctx.amgt_set_source_iso(prob["q"])
    for f, (kind, val) in enumerate(prob["boundary"]):
        ctx.amgt_set_boundary(f, kind, val)
    return ctx
