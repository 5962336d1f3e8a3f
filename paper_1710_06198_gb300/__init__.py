"""Python binding of libtmg, the GB300 twisted-mass DD-alpha-AMG library (arXiv:1710.06198).

Argument marshalling only: every operation runs in the library's CUDA kernels through the C ABI
declared in ``include/tmg.h``.  Arrays are complex128 in lexicographic site order
(``[..., T, Z, Y, X, 4, 3]`` for spinors, ``[T, Z, Y, X, 4, 3, 3]`` for links, ``[..., Vc, 2 Nv]``
for coarse vectors).  numpy arrays are passed as host memory; CUDA torch tensors (complex128) are
passed as device memory on the context's device, and the call is ordered on the context stream.

The library is loaded from this directory (``libtmg.so``, built by ``build.py``).  If it is
missing, :func:`lib` raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtmg.so")

PREC_F64, PREC_F32, PREC_F16 = 0, 1, 2
HOST, DEVICE = 0, 1
OP_D, OP_DDAG, OP_DND, OP_HOP, OP_DHAT, OP_DHAT_DAG = 0, 1, 2, 3, 4, 5
SOLVE_MG_F64, SOLVE_MG_MIXED, SOLVE_CG_F64, SOLVE_MG_BATCHED = 0, 1, 2, 3
SOLVE_ND_F64, SOLVE_ND_MIXED, SOLVE_CG_EO = 4, 5, 6
STATUS = {0: "TMG_OK", -1: "TMG_ERR_ARG", -2: "TMG_ERR_CUDA", -3: "TMG_ERR_OOM", -4: "TMG_ERR_NOCONV",
          -5: "TMG_ERR_BREAKDOWN", -6: "TMG_ERR_TIMEOUT", -7: "TMG_ERR_STATE"}

_lib = None


class TmgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class MGParams(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int), ("sap_sweeps", ctypes.c_int), ("sap_mr", ctypes.c_int),
                ("coarse_m", ctypes.c_int), ("coarse_rtol", ctypes.c_double), ("n_init", ctypes.c_int),
                ("n_iter", ctypes.c_int), ("restart", ctypes.c_int), ("prec_fine", ctypes.c_int),
                ("prec_coarse", ctypes.c_int)]


class Level2Params(ctypes.Structure):
    _fields_ = [("agg", ctypes.c_int * 4), ("nv", ctypes.c_int), ("smooth_m", ctypes.c_int),
                ("k_restart", ctypes.c_int), ("k_rtol", ctypes.c_double), ("coarse_m", ctypes.c_int),
                ("coarse_rtol", ctypes.c_double), ("n_init", ctypes.c_int), ("n_iter", ctypes.c_int)]


class HmcParams(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("tau", ctypes.c_double), ("n_mono", ctypes.c_int),
                ("mu", ctypes.c_double * 8), ("mu2", ctypes.c_double * 8), ("level", ctypes.c_int * 8),
                ("n_levels", ctypes.c_int), ("steps", ctypes.c_int * 8), ("tol_action", ctypes.c_double),
                ("tol_force", ctypes.c_double), ("setup_iters_start", ctypes.c_int),
                ("setup_iters_force", ctypes.c_int), ("keep_phi", ctypes.c_int)]


class HmcStats(ctypes.Structure):
    _fields_ = [("H_start", ctypes.c_double), ("H_end", ctypes.c_double), ("solves", ctypes.c_longlong),
                ("outer_iterations", ctypes.c_longlong), ("fermion_forces", ctypes.c_longlong),
                ("gauge_forces", ctypes.c_longlong), ("link_updates", ctypes.c_longlong),
                ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("refinements", ctypes.c_int), ("coarse_iterations", ctypes.c_int),
                ("true_residual", ctypes.c_double), ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P, _I, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
_SIGS = {
    "tmg_create": [ctypes.POINTER(_P), _P, _P, _I, _P],
    "tmg_destroy": [_P],
    "tmg_last_error": [_P],
    "tmg_version": [],
    "tmg_load_gauge": [_P, _P, _I, _I],
    "tmg_set_params": [_P, _D, _D, _D, _D, _D],
    "tmg_apply": [_P, _I, _P, _P, _I, _P, _I, _I],
    "tmg_mg_defaults": [ctypes.POINTER(MGParams)],
    "tmg_setup": [_P, ctypes.POINTER(MGParams), _P, _I],
    "tmg_get_vectors": [_P, _P, _I],
    "tmg_sap": [_P, _P, _P, _I, _I],
    "tmg_restrict": [_P, _P, _P, _I, _I],
    "tmg_prolong": [_P, _P, _P, _I, _I],
    "tmg_coarse_apply": [_P, _P, _P, _D, _I, _I],
    "tmg_cycle": [_P, _P, _P, _I],
    "tmg_coarse_solve": [_P, _P, _P, _D, _I, _I],
    "tmg_coarse_apply_multi": [_P, _P, _P, _I, _P, _I],
    "tmg_coarse_solve_multi": [_P, _P, _P, _I, _P, _I],
    "tmg_kcycle_multi": [_P, _P, _P, _I, _P, _I, _I],
    "tmg_coarse_solve_noalloc": [_P, _P, _P, _D, _I],
    "tmg_solve": [_P, _P, _P, _I, _P, _D, _I, _I, ctypes.POINTER(Stats), _I],
    "tmg_bench_dslash": [_P, _I, _I, ctypes.POINTER(_D)],
    "tmg_launch_count": [_P, ctypes.POINTER(ctypes.c_longlong)],
    "tmg_profile": [_P, _I],
    "tmg_tune": [_P, ctypes.c_char_p, _D],
    "tmg_force_xy": [_P, _P, _P, _P, _I],
    "tmg_force": [_P, _P, _P, _D, ctypes.POINTER(_D), ctypes.POINTER(Stats), _I],
    "tmg_profile_read": [_P, _I, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_D)],
    "tmg_level2_defaults": [ctypes.POINTER(Level2Params)],
    "tmg_setup_level2": [_P, ctypes.POINTER(Level2Params), _P, _I],
    "tmg_get_vectors2": [_P, _P, _I],
    "tmg_restrict2": [_P, _P, _P, _I, _I],
    "tmg_prolong2": [_P, _P, _P, _I, _I],
    "tmg_coarse_apply2": [_P, _P, _P, _D, _I, _I],
    "tmg_kcycle": [_P, _P, _P, _D, _I, _I, _I],
    "tmg_sap_nd": [_P, _P, _P, _I, _I],
    "tmg_coarse_apply_nd": [_P, _P, _P, _I, _I],
    "tmg_coarse_solve_nd": [_P, _P, _P, _I, _I],
    "tmg_kcycle_nd": [_P, _P, _P, _I, _I, _I],
    "tmg_cycle_nd": [_P, _P, _P, _I],
    "tmg_autotune": [_P, ctypes.POINTER(_D)],
    "tmg_graph_count": [_P, ctypes.POINTER(_I)],
    "tmg_rotate_gauge": [_P, _P, _D, _I],
    "tmg_setup_update": [_P, _I],
    "tmg_pf_action": [_P, _P, _P, _D, ctypes.POINTER(_D), ctypes.POINTER(Stats), _I],
    "tmg_pf_force": [_P, _P, _P, _D, ctypes.POINTER(Stats), _I],
    "tmg_sigma_min": [_P, _P, _D, _I, _D, _D, _I, ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_I), _I],
    "tmg_solve_shifts": [_P, _P, _P, _I, _P, _D, _I, _D, _P, ctypes.POINTER(Stats), _I],
    "tmg_bench_schur": [_P, _I, _I, ctypes.POINTER(_D)],
    "tmg_mms_cg": [_P, _P, _P, _I, _P, _D, _I, ctypes.POINTER(Stats), _I],
    "tmg_rational_apply": [_P, _P, _P, _I, _D, _P, _P, _D, _I, _D, ctypes.POINTER(Stats), _I],
    "tmg_set_ndshift": [_P, _D],
    "tmg_hmc_trajectory": [_P, ctypes.POINTER(HmcParams), _P, _P, ctypes.POINTER(_D), ctypes.POINTER(HmcStats), _I],
    "tmg_get_gauge": [_P, _P, _I],
    "tmg_gauge_action": [_P, _D, ctypes.POINTER(_D)],
    "tmg_gauge_force": [_P, _D, _P, _I],
    "tmg_check_links": [_P, ctypes.c_longlong, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_longlong)],
}

PROFILE_KINDS = ["dslash_f64", "dslash_f32", "dslash_f16", "sap_f64", "sap_f32", "sap_f16", "restrict",
                 "prolong", "coarse_apply", "coarse_solve", "eo_f64", "eo_f32"]


def lib():
    """Load libtmg.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError(f"libtmg.so not built ({LIB_PATH}); run paper_1710_06198_gb300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_char_p if name in ("tmg_last_error", "tmg_version") else ctypes.c_int
        _lib = L
    return _lib


def _is_torch_cuda(a):
    return type(a).__module__.startswith("torch") and getattr(a, "is_cuda", False)


def _ptr(a):
    """(pointer, where) of a complex128 numpy array or CUDA torch tensor."""
    if _is_torch_cuda(a):
        import torch
        if a.dtype != torch.complex128 or not a.is_contiguous():
            raise TypeError("device arrays must be contiguous complex128 torch tensors")
        return ctypes.c_void_p(a.data_ptr()), DEVICE
    if not isinstance(a, np.ndarray) or a.dtype != np.complex128 or not a.flags.c_contiguous:
        raise TypeError("host arrays must be C-contiguous complex128 numpy arrays")
    return ctypes.c_void_p(a.ctypes.data), HOST


def _ptr_real(a):
    """(pointer, where) of a float64 numpy array or CUDA torch tensor."""
    if _is_torch_cuda(a):
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("device arrays must be contiguous float64 torch tensors")
        return ctypes.c_void_p(a.data_ptr()), DEVICE
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags.c_contiguous:
        raise TypeError("host arrays must be C-contiguous float64 numpy arrays")
    return ctypes.c_void_p(a.ctypes.data), HOST


def _empty_real_like(a, shape):
    if _is_torch_cuda(a):
        import torch
        return torch.empty(shape, dtype=torch.float64, device=a.device)
    return np.empty(shape, dtype=np.float64)


def _empty_like(a, shape):
    if _is_torch_cuda(a):
        import torch
        return torch.empty(shape, dtype=torch.complex128, device=a.device)
    return np.empty(shape, dtype=np.complex128)


def _same_where(*arrays):
    wh = {_ptr(a)[1] for a in arrays}
    if len(wh) != 1:
        raise TypeError("mixing host and device arrays in one call")


@dataclass
class OperatorParams:
    kappa: float
    csw: float = 0.0
    mu: float = 0.0
    mubar: float = 0.0
    epsbar: float = 0.0


class Context:
    """One lattice on one GPU: gauge field, operator parameters and multigrid hierarchy."""

    def __init__(self, dims, block, device=0, stream=None):
        self.dims = tuple(int(d) for d in dims)
        self.block = tuple(int(b) for b in block)
        self.lat = (self.dims[3], self.dims[2], self.dims[1], self.dims[0])
        self.V = int(np.prod(self.dims))
        self.coarse_lat = tuple(self.lat[i] // self.block[3 - i] for i in range(4))
        self.nv = None
        h = ctypes.c_void_p()
        d = (ctypes.c_int * 4)(*self.dims)
        b = (ctypes.c_int * 4)(*self.block)
        st = ctypes.c_void_p(stream) if stream is not None else None
        rc = lib().tmg_create(ctypes.byref(h), d, b, int(device), st)
        if rc != 0:
            raise TmgError(rc, "tmg_create rejected the geometry or device")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().tmg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, rc):
        if rc != 0:
            raise TmgError(rc, lib().tmg_last_error(self._h).decode())

    # ---- operator data
    def load_gauge(self, U, t_bc=-1):
        p, wh = _ptr(U)
        self._check(lib().tmg_load_gauge(self._h, p, wh, int(t_bc)))
        self.gauge_version = getattr(self, "gauge_version", 0) + 1

    @staticmethod
    def hmc_params(beta, tau, monomials, steps, tol_action=1e-11, tol_force=1e-9, setup_iters_start=3,
                   setup_iters_force=1, keep_phi=False):
        """monomials: list of (mu, mu2 or 0, level); steps: minimal-norm steps per call of each time
        scale (the gauge action on the last)."""
        hp = HmcParams()
        hp.beta, hp.tau, hp.n_mono, hp.n_levels = float(beta), float(tau), len(monomials), len(steps)
        for i, (m, m2, lv) in enumerate(monomials):
            hp.mu[i], hp.mu2[i], hp.level[i] = float(m), float(m2), int(lv)
        for i, n in enumerate(steps):
            hp.steps[i] = int(n)
        hp.tol_action, hp.tol_force = float(tol_action), float(tol_force)
        hp.setup_iters_start, hp.setup_iters_force, hp.keep_phi = int(setup_iters_start), int(setup_iters_force), int(keep_phi)
        return hp

    def hmc_trajectory(self, params, P, eta):
        """(dH, stats): one trajectory; P (float64 [T, Z, Y, X, 4, 8]) is updated in place, eta
        (complex128 [n_mono, T, Z, Y, X, 4, 3]) feeds the heat bath; the context keeps the new field."""
        pp, wh = _ptr_real(P)
        pe, we = _ptr(eta)
        if wh != we:
            raise TypeError("P and eta must both be host or both device arrays")
        dH, st = ctypes.c_double(), HmcStats()
        self._check(lib().tmg_hmc_trajectory(self._h, ctypes.byref(params), pp, pe, ctypes.byref(dH), ctypes.byref(st), wh))
        self.gauge_version = getattr(self, "gauge_version", 0) + 1
        return dH.value, st.as_dict()

    def get_gauge(self, like=None):
        U = _empty_like(like, self.lat + (4, 3, 3)) if like is not None else np.empty(self.lat + (4, 3, 3), np.complex128)
        p, wh = _ptr(U)
        self._check(lib().tmg_get_gauge(self._h, p, wh))
        return U

    def gauge_action(self, beta):
        S = ctypes.c_double()
        self._check(lib().tmg_gauge_action(self._h, float(beta), ctypes.byref(S)))
        return S.value

    def gauge_force(self, beta):
        f = np.empty(self.lat + (4, 8), np.float64)
        p, wh = _ptr_real(f)
        self._check(lib().tmg_gauge_force(self._h, float(beta), p, wh))
        return f

    def set_ndshift(self, delta):
        """Doublet operators become D_ND + i delta (G5 x tau1) (the shifted systems of Sec. 3)."""
        self._check(lib().tmg_set_ndshift(self._h, float(delta)))

    def rotate_gauge(self, omega, step=1.0):
        """U_mu(x) <- exp(i step omega(x, mu) . lambda / 2) U_mu(x); omega float64 [T, Z, Y, X, 4, 8]."""
        p, wh = _ptr_real(omega)
        self._check(lib().tmg_rotate_gauge(self._h, p, float(step), wh))
        self.gauge_version = getattr(self, "gauge_version", 0) + 1

    def setup_update(self, n_iter=1):
        """Refine the last setup's test vectors by n_iter cycle iterations on the current field."""
        self._check(lib().tmg_setup_update(self._h, int(n_iter)))

    def pf_action(self, phi, tol=1e-10):
        """(S, Y, stats): S = ||D^-1 phi||^2 and the solution Y = D^-1 phi."""
        Y = _empty_like(phi, phi.shape)
        pp, wh = _ptr(phi)
        py, _ = _ptr(Y)
        S = ctypes.c_double()
        st = Stats()
        self._check(lib().tmg_pf_action(self._h, pp, py, float(tol), ctypes.byref(S), ctypes.byref(st), wh))
        return S.value, Y, st.as_dict()

    def pf_force(self, Y, tol=1e-10):
        """(f, stats): su(3) force coefficients f[T, Z, Y, X, 4, 8] of S from its solution Y."""
        f = _empty_real_like(Y, self.lat + (4, 8))
        py, wh = _ptr(Y)
        pf, _ = _ptr_real(f)
        st = Stats()
        self._check(lib().tmg_pf_force(self._h, py, pf, float(tol), ctypes.byref(st), wh))
        return f, st.as_dict()

    def sigma_min(self, start, mu_s, max_steps=40, rtol=1e-4, solve_tol=1e-9, method=SOLVE_MG_F64, check=True):
        """(sigma, ritz_residual, solves): sigma_min(D_W) by Lanczos on (D(mu_s)^dag D(mu_s))^-1."""
        ps, wh = _ptr(start)
        sg, rr, ns = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        rc = lib().tmg_sigma_min(self._h, ps, float(mu_s), int(max_steps), float(rtol), float(solve_tol), int(method),
                                 ctypes.byref(sg), ctypes.byref(rr), ctypes.byref(ns), wh)
        if check and rc != -4:
            self._check(rc)
        return sg.value, rr.value, ns.value

    def set_params(self, kappa, csw=0.0, mu=0.0, mubar=0.0, epsbar=0.0):
        self._check(lib().tmg_set_params(self._h, kappa, csw, mu, mubar, epsbar))

    def apply(self, x, op=OP_D, prec=PREC_F64, mu_per_col=None):
        """y = op x for x[..., T, Z, Y, X, 4, 3] (TMG_OP_DND: x[..., 2, T, Z, Y, X, 4, 3])."""
        per = 2 * self.V * 12 if op == OP_DND else self.V * 12
        n = int(np.prod(x.shape)) // per
        y = _empty_like(x, x.shape)
        px, wh = _ptr(x)
        py, _ = _ptr(y)
        mp = None
        if mu_per_col is not None:
            mu_arr = np.ascontiguousarray(np.asarray(mu_per_col, dtype=np.float64).reshape(n))
            mp = mu_arr.ctypes.data_as(ctypes.c_void_p)
        self._check(lib().tmg_apply(self._h, op, px, py, n, mp, prec, wh))
        return y

    # ---- multigrid
    @staticmethod
    def mg_defaults():
        p = MGParams()
        lib().tmg_mg_defaults(ctypes.byref(p))
        return p

    def setup(self, v0, params: MGParams):
        _same_where(v0)
        p, wh = _ptr(v0)
        self._check(lib().tmg_setup(self._h, ctypes.byref(params), p, wh))
        self.nv = params.nv

    def get_vectors(self, like=None):
        shape = (self.nv,) + self.lat + (4, 3)
        W = _empty_like(like, shape) if like is not None else np.empty(shape, np.complex128)
        p, wh = _ptr(W)
        self._check(lib().tmg_get_vectors(self._h, p, wh))
        return W

    def sap(self, b, x0, prec=PREC_F64):
        x = x0.copy() if not _is_torch_cuda(x0) else x0.clone()
        pb, wh = _ptr(b)
        px, _ = _ptr(x)
        self._check(lib().tmg_sap(self._h, pb, px, prec, wh))
        return x

    def restrict(self, r, prec=PREC_F64):
        c = _empty_like(r, self.coarse_lat + (2 * self.nv,))
        pr, wh = _ptr(r)
        pc, _ = _ptr(c)
        self._check(lib().tmg_restrict(self._h, pr, pc, prec, wh))
        return c

    def prolong(self, c, prec=PREC_F64):
        e = _empty_like(c, self.lat + (4, 3))
        pc, wh = _ptr(c)
        pe, _ = _ptr(e)
        self._check(lib().tmg_prolong(self._h, pc, pe, prec, wh))
        return e

    def coarse_apply(self, x, mu=0.0, prec=PREC_F64):
        y = _empty_like(x, x.shape)
        px, wh = _ptr(x)
        py, _ = _ptr(y)
        self._check(lib().tmg_coarse_apply(self._h, px, py, float(mu), prec, wh))
        return y

    def coarse_apply_multi(self, x, mu_per_col=None):
        """Y[n] = D_c(mu_n) X[n] for x[n_rhs, ..., 2 Nv] on the tensor cores."""
        n = x.shape[0]
        y = _empty_like(x, x.shape)
        px, wh = _ptr(x)
        py, _ = _ptr(y)
        mp = None
        if mu_per_col is not None:
            mu_arr = np.ascontiguousarray(np.asarray(mu_per_col, dtype=np.float64).reshape(n))
            mp = mu_arr.ctypes.data_as(ctypes.c_void_p)
        self._check(lib().tmg_coarse_apply_multi(self._h, px, py, n, mp, wh))
        return y

    def coarse_solve_multi(self, b, mu_per_col=None):
        """X[n] ~= D_c(mu_n)^-1 B[n] for b[n_rhs, ..., 2 Nv]: the batched coarse GMRES (FP32)."""
        n = b.shape[0]
        x = _empty_like(b, b.shape)
        pb, wh = _ptr(b)
        px, _ = _ptr(x)
        mp = None
        if mu_per_col is not None:
            mu_arr = np.ascontiguousarray(np.asarray(mu_per_col, dtype=np.float64).reshape(n))
            mp = mu_arr.ctypes.data_as(ctypes.c_void_p)
        self._check(lib().tmg_coarse_solve_multi(self._h, pb, px, n, mp, wh))
        return x

    def coarse_solve(self, c, mu=0.0, prec=PREC_F64):
        """x ~= D_c(mu)^-1 c by the coarse GMRES of the cycle."""
        x = _empty_like(c, c.shape)
        pc, wh = _ptr(c)
        px, _ = _ptr(x)
        self._check(lib().tmg_coarse_solve(self._h, pc, px, float(mu), prec, wh))
        return x

    # ---- third level
    @staticmethod
    def level2_defaults():
        p = Level2Params()
        lib().tmg_level2_defaults(ctypes.byref(p))
        return p

    def setup_level2(self, v1, params: Level2Params):
        """Level-2 setup on D_c from nv level-1 vectors v1[nv, ..., 2 Nv]."""
        _same_where(v1)
        p, wh = _ptr(v1)
        self._check(lib().tmg_setup_level2(self._h, ctypes.byref(params), p, wh))
        self.nv2 = params.nv
        self.agg2 = tuple(params.agg)

    @property
    def coarse2_lat(self):
        """Level-2 lattice as (T, Z, Y, X)."""
        c = self.coarse_lat
        a = self.agg2
        return (c[0] // a[3], c[1] // a[2], c[2] // a[1], c[3] // a[0])

    def get_vectors2(self, like=None):
        shape = (self.nv2,) + self.coarse_lat + (2 * self.nv,)
        W = _empty_like(like, shape) if like is not None else np.empty(shape, np.complex128)
        p, wh = _ptr(W)
        self._check(lib().tmg_get_vectors2(self._h, p, wh))
        return W

    def restrict2(self, c, prec=PREC_F64):
        c2 = _empty_like(c, self.coarse2_lat + (2 * self.nv2,))
        pc, wh = _ptr(c)
        p2, _ = _ptr(c2)
        self._check(lib().tmg_restrict2(self._h, pc, p2, prec, wh))
        return c2

    def prolong2(self, c2, prec=PREC_F64):
        e = _empty_like(c2, self.coarse_lat + (2 * self.nv,))
        p2, wh = _ptr(c2)
        pe, _ = _ptr(e)
        self._check(lib().tmg_prolong2(self._h, p2, pe, prec, wh))
        return e

    def coarse_apply2(self, x, mu=0.0, prec=PREC_F64):
        y = _empty_like(x, x.shape)
        px, wh = _ptr(x)
        py, _ = _ptr(y)
        self._check(lib().tmg_coarse_apply2(self._h, px, py, float(mu), prec, wh))
        return y

    def kcycle(self, b, mu=0.0, mode=0, prec=PREC_F64):
        """Level-1 K-cycle kernel: mode 0 solve, 1 level-1 cycle, 2 smoother from zero."""
        x = _empty_like(b, b.shape)
        pb, wh = _ptr(b)
        px, _ = _ptr(x)
        self._check(lib().tmg_kcycle(self._h, pb, px, float(mu), int(mode), prec, wh))
        return x

    def kcycle_multi(self, b, mu_per_col=None, mode=0):
        """The K-cycle (FP32) on b[n_rhs, ..., 2 Nv] in lock-step, column n with twist mu_per_col[n]."""
        n = b.shape[0]
        x = _empty_like(b, b.shape)
        pb, wh = _ptr(b)
        px, _ = _ptr(x)
        mp = None
        if mu_per_col is not None:
            mu_arr = np.ascontiguousarray(np.asarray(mu_per_col, dtype=np.float64).reshape(n))
            mp = mu_arr.ctypes.data_as(ctypes.c_void_p)
        self._check(lib().tmg_kcycle_multi(self._h, pb, px, n, mp, int(mode), wh))
        return x

    # ---- non-degenerate doublet (flavour pairs: fine [2, ..., 4, 3], coarse [2, ..., 2 Nv])
    def sap_nd(self, b2, x2, prec=PREC_F64):
        x = x2.copy() if not _is_torch_cuda(x2) else x2.clone()
        pb, wh = _ptr(b2)
        px, _ = _ptr(x)
        self._check(lib().tmg_sap_nd(self._h, pb, px, prec, wh))
        return x

    def _coarse_nd(self, fn, x2, *extra):
        y = _empty_like(x2, x2.shape)
        px, wh = _ptr(x2)
        py, _ = _ptr(y)
        self._check(fn(self._h, px, py, *extra, wh))
        return y

    def coarse_apply_nd(self, x2, prec=PREC_F64):
        return self._coarse_nd(lib().tmg_coarse_apply_nd, x2, prec)

    def coarse_solve_nd(self, b2, prec=PREC_F64):
        return self._coarse_nd(lib().tmg_coarse_solve_nd, b2, prec)

    def kcycle_nd(self, b2, mode=0, prec=PREC_F64):
        return self._coarse_nd(lib().tmg_kcycle_nd, b2, int(mode), prec)

    def cycle_nd(self, r2):
        z = _empty_like(r2, r2.shape)
        pr, wh = _ptr(r2)
        pz, _ = _ptr(z)
        self._check(lib().tmg_cycle_nd(self._h, pr, pz, wh))
        return z

    def cycle(self, r):
        z = _empty_like(r, r.shape)
        pr, wh = _ptr(r)
        pz, _ = _ptr(z)
        self._check(lib().tmg_cycle(self._h, pr, pz, wh))
        return z

    def solve(self, b, tol=1e-10, method=SOLVE_MG_MIXED, maxiter=10000, mu_per_col=None, out=None,
              check=True):
        n = int(np.prod(b.shape)) // (self.V * 12)
        if method in (SOLVE_ND_F64, SOLVE_ND_MIXED):
            n //= 2                                   # flavour pairs
        x = _empty_like(b, b.shape) if out is None else out
        pb, wh = _ptr(b)
        px, _ = _ptr(x)
        st = Stats()
        mp = None
        if mu_per_col is not None:
            mu_arr = np.ascontiguousarray(np.asarray(mu_per_col, dtype=np.float64).reshape(n))
            mp = mu_arr.ctypes.data_as(ctypes.c_void_p)
        rc = lib().tmg_solve(self._h, pb, px, n, mp, float(tol), int(method), int(maxiter), ctypes.byref(st), wh)
        if check:
            self._check(rc)
        return x, st.as_dict()

    def solve_shifts(self, b, mus, tol=1e-10, guess=2, taylor_tol=1e-2):
        """(x[n_shift, ...], per-system outer iterations, stats) for D(mu_k) x_k = b in order, with zero
        (0), previous-solution (1) or first-order Taylor (2) initial guesses."""
        mu_arr = np.ascontiguousarray(np.asarray(mus, dtype=np.float64).reshape(-1))
        n = mu_arr.size
        x = _empty_like(b, (n,) + tuple(b.shape))
        pb, wh = _ptr(b)
        px, _ = _ptr(x)
        its = (ctypes.c_int * n)()
        st = Stats()
        self._check(lib().tmg_solve_shifts(self._h, pb, px, n, mu_arr.ctypes.data_as(ctypes.c_void_p), float(tol),
                                           int(guess), float(taylor_tol), its, ctypes.byref(st), wh))
        return x, list(its), st.as_dict()

    def mms_cg(self, b, sigma, tol=1e-10, flavours=1):
        """(x[n_shift, ...], stats): (A + sigma_s)^-1 b for all shifts, A = D^dag D or Q_ND^2."""
        sg = np.ascontiguousarray(np.asarray(sigma, dtype=np.float64).reshape(-1))
        x = _empty_like(b, (sg.size,) + tuple(b.shape))
        pb, wh = _ptr(b)
        px, _ = _ptr(x)
        st = Stats()
        self._check(lib().tmg_mms_cg(self._h, pb, px, sg.size, sg.ctypes.data_as(ctypes.c_void_p), float(tol),
                                     int(flavours), ctypes.byref(st), wh))
        return x, st.as_dict()

    def rational_apply(self, phi, a, num, den, tol=1e-10, flavours=1, mg_below=0.0):
        """(a prod (A + num_l)/(A + den_l) phi, stats): shifts >= mg_below by the multi-shift CG, the
        smaller ones by the multigrid (two solves each)."""
        nu = np.ascontiguousarray(np.asarray(num, dtype=np.float64).reshape(-1))
        de = np.ascontiguousarray(np.asarray(den, dtype=np.float64).reshape(-1))
        out = _empty_like(phi, phi.shape)
        pp, wh = _ptr(phi)
        po, _ = _ptr(out)
        st = Stats()
        self._check(lib().tmg_rational_apply(self._h, pp, po, nu.size, float(a), nu.ctypes.data_as(ctypes.c_void_p),
                                             de.ctypes.data_as(ctypes.c_void_p), float(tol), int(flavours),
                                             float(mg_below), ctypes.byref(st), wh))
        return out, st.as_dict()

    def force_xy(self, X, Y):
        """F[T, Z, Y, X, mu, 3, 3] of S = ||D^-1 phi||^2 from X = D^-dag Y, Y = D^-1 phi."""
        F = _empty_like(X, self.lat + (4, 3, 3))
        px, wh = _ptr(X)
        py, _ = _ptr(Y)
        pf, _ = _ptr(F)
        self._check(lib().tmg_force_xy(self._h, px, py, pf, wh))
        return F

    def force(self, phi, tol=1e-10):
        """(S, F, stats): action and force with both solves done by the multigrid."""
        F = _empty_like(phi, self.lat + (4, 3, 3))
        pp, wh = _ptr(phi)
        pf, _ = _ptr(F)
        S = ctypes.c_double()
        st = Stats()
        self._check(lib().tmg_force(self._h, pp, pf, float(tol), ctypes.byref(S), ctypes.byref(st), wh))
        return S.value, F, st.as_dict()

    def autotune(self):
        """Pick the fastest launch shape of the coarse solve; returns its time per solve in ms."""
        ms = ctypes.c_double()
        self._check(lib().tmg_autotune(self._h, ctypes.byref(ms)))
        return ms.value

    def tune(self, key, value):
        self._check(lib().tmg_tune(self._h, key.encode(), float(value)))

    def bench_schur(self, prec=PREC_F32, n_iter=100):
        """Mean milliseconds per application of the even-odd reduced operator (two kernels)."""
        ms = ctypes.c_double()
        self._check(lib().tmg_bench_schur(self._h, prec, n_iter, ctypes.byref(ms)))
        return ms.value

    def bench_dslash(self, prec=PREC_F32, n_iter=100):
        ms = ctypes.c_double()
        self._check(lib().tmg_bench_dslash(self._h, prec, n_iter, ctypes.byref(ms)))
        return ms.value


def profile(ctx: "Context", enable: bool):
    ctx._check(lib().tmg_profile(ctx._h, int(bool(enable))))


def profile_read(ctx: "Context"):
    """{kind: (launches, total ms)} of the kernel classes timed since profile(ctx, True)."""
    out = {}
    for k, name in enumerate(PROFILE_KINDS):
        n, ms = ctypes.c_longlong(), ctypes.c_double()
        ctx._check(lib().tmg_profile_read(ctx._h, k, ctypes.byref(n), ctypes.byref(ms)))
        out[name] = (n.value, ms.value)
    return out


def launch_count(ctx: "Context"):
    n = ctypes.c_longlong()
    ctx._check(lib().tmg_launch_count(ctx._h, ctypes.byref(n)))
    return n.value


def graph_count(ctx: "Context"):
    n = ctypes.c_int()
    ctx._check(lib().tmg_graph_count(ctx._h, ctypes.byref(n)))
    return n.value


def version():
    return lib().tmg_version().decode()


def check_links(U):
    """(ok, worst defect, index of the worst link) of a host field of SU(3) links [..., 3, 3]
    (complex128); runs on the host, needs no GPU."""
    if not isinstance(U, np.ndarray) or U.dtype != np.complex128 or not U.flags.c_contiguous:
        raise TypeError("host arrays must be C-contiguous complex128 numpy arrays")
    w, i = ctypes.c_double(), ctypes.c_longlong()
    rc = lib().tmg_check_links(ctypes.c_void_p(U.ctypes.data), U.size // 9, ctypes.byref(w), ctypes.byref(i))
    return rc == 0, w.value, i.value
