"""Thin ctypes binding of liboverlap (include/overlap.h): argument marshalling only.

Every function keeps its C name. Spinor arguments may be numpy arrays (host
memory, on_device = 0) or torch CUDA tensors (device memory, on_device = 1) of
complex128 or complex64 in the canonical layout [..., Lt, Lz, Ly, Lx, 4, 3]; all
arithmetic happens in the library. A missing or unloadable library raises
immediately; there is no fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("OVL_LIB_PATH", os.path.join(_HERE, "liboverlap.so"))

OVL_OK, OVL_EINVAL, OVL_ENOMEM, OVL_ECUDA, OVL_ENOCONV, OVL_EBREAKDOWN, OVL_EAPPROX, OVL_ETIMEOUT = \
    0, -1, -2, -3, -4, -5, -6, -7
OVL_C128, OVL_C64 = 0, 1
OVL_PREC_F64, OVL_PREC_F32, OVL_PREC_F16, OVL_PREC_F64E, OVL_PREC_AUTO = 0, 1, 2, 3, -1
OVL_SOLVER_SUMR, OVL_SOLVER_CG = 0, 1
OVL_PROF_CLASSES = 9
PROF_NAMES = ["wilson_f64", "wilson_f32", "wilson_f16", "mscg_update", "vector", "scalar", "gram", "force",
              "wilson_f64e"]

STATUS_NAMES = {0: "OVL_OK", -1: "OVL_EINVAL", -2: "OVL_ENOMEM", -3: "OVL_ECUDA", -4: "OVL_ENOCONV",
                -5: "OVL_EBREAKDOWN", -6: "OVL_EAPPROX", -7: "OVL_ETIMEOUT"}


class OvlError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class ovl_params(ctypes.Structure):
    _fields_ = [("solver", ctypes.c_int), ("mixed", ctypes.c_int), ("half_storage", ctypes.c_int),
                ("emulate_fp64", ctypes.c_int),
                ("eta_floor", ctypes.c_double), ("sp_switch", ctypes.c_double), ("half_switch", ctypes.c_double),
                ("eta_precond", ctypes.c_double), ("relax_factor", ctypes.c_double),
                ("gmresr_max", ctypes.c_int), ("inner_max", ctypes.c_int), ("mscg_max", ctypes.c_int),
                ("delta_split", ctypes.c_double), ("c_spec", ctypes.c_double), ("bc_t", ctypes.c_int),
                ("a_override", ctypes.c_double), ("b_override", ctypes.c_double), ("batch_max", ctypes.c_int), ("wilson_variant", ctypes.c_int),
                ("use_graphs", ctypes.c_int),
                ("verify", ctypes.c_int), ("sign_method", ctypes.c_int), ("basis_gb", ctypes.c_double),
                ("multimass", ctypes.c_int), ("force_pole_group", ctypes.c_int), ("lanczos_cap", ctypes.c_int),
                ("gram_method", ctypes.c_int),
                ("stream", ctypes.c_void_p)]


class ovl_solve_info(ctypes.Structure):
    _fields_ = [("converged", ctypes.c_int), ("outer_iters", ctypes.c_int), ("inner_iters", ctypes.c_int),
                ("sign_calls", ctypes.c_int), ("wilson_calls", ctypes.c_longlong),
                ("wilson_f64", ctypes.c_longlong), ("wilson_f32", ctypes.c_longlong),
                ("wilson_f16", ctypes.c_longlong), ("true_residual", ctypes.c_double), ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
P = ctypes.c_void_p
I = ctypes.c_int
D = ctypes.c_double
DP = ctypes.POINTER(ctypes.c_double)
LLP = ctypes.POINTER(ctypes.c_longlong)

_SIGS = {
    "ovl_version": (ctypes.c_char_p, []),
    "ovl_params_default": (I, [ctypes.POINTER(ovl_params)]),
    "ovl_zolotarev_coeffs": (I, [I, D, D, DP, DP, DP]),
    "ovl_host_eigh": (I, [I, DP, DP, DP]),
    "ovl_host_cholesky": (I, [I, DP, DP]),
    "ovl_host_lower_inverse": (I, [I, DP, DP]),
    "ovl_host_lu_solve": (I, [I, DP, DP, I, DP]),
    "ovl_host_tridiag_extremes": (I, [I, DP, DP, DP, DP]),
    "ovl_host_ritz": (I, [I, DP, DP, DP, D, D, I, I, DP, DP, DP, ctypes.POINTER(I)]),
    "ovl_host_sumr_step": (I, [D, DP, DP, DP]),
    "ovl_host_defl_start": (I, [I, DP, DP, DP, DP, DP, I, DP, DP, DP, I, DP]),
    "ovl_host_rayleigh_ritz": (I, [I, DP, DP, DP, DP]),
    "overlap_create": (I, [ctypes.POINTER(P), ctypes.POINTER(I), DP, D, D, I, D, ctypes.POINTER(ovl_params)]),
    "overlap_destroy": (None, [P]),
    "overlap_last_error": (ctypes.c_char_p, [P]),
    "ovl_trim": (I, [P]),
    "overlap_zolotarev": (I, [P, DP, DP, DP, DP, DP]),
    "ovl_wilson_apply": (I, [P, P, P, I, I, I, I]),
    "ovl_wilson_apply_noalloc": (I, [P, P, P, I, I, I]),
    "ovl_sign_apply": (I, [P, P, P, I, I, I, D, I]),
    "overlap_apply": (I, [P, D, P, P, I, I, I, D, I, I]),
    "overlap_sumr": (I, [P, D, P, P, I, I, I, D, D, I, DP, ctypes.POINTER(I)]),
    "overlap_solve": (I, [P, I, DP, I, P, P, I, I, D, P, ctypes.POINTER(ovl_solve_info)]),
    "eigsumr_accumulate": (I, [P, ctypes.POINTER(P), I, I, D, P, P, I, I, D, ctypes.POINTER(ovl_solve_info)]),
    "ovl_defl_info": (I, [P, ctypes.POINTER(I), DP, DP]),
    "ovl_ritz_recalculate": (I, [P, I, I, D, D, P, P, P, P, I, I, DP, DP]),
    "ovl_eigensolve": (I, [P, ctypes.POINTER(P), I, I, D, P, I, I, I, D, I, ctypes.POINTER(I)]),
    "ovl_defl_vector": (I, [P, I, DP, DP]),
    "ovl_defl_save": (I, [P, ctypes.c_char_p]),
    "ovl_defl_load": (I, [P, ctypes.POINTER(P), ctypes.c_char_p]),
    "ovl_defl_destroy": (None, [P]),
    "overlap_force": (I, [P, D, P, I, I, D, DP, DP]),
    "ovl_profile_enable": (I, [P, I]),
    "ovl_profile_reset": (I, [P]),
    "ovl_profile_get": (I, [P, I, LLP, DP, DP]),
    "ovl_profile_units": (I, [P, I, DP]),
    "ovl_bench_wilson": (I, [P, I, I, I, DP, DP]),
    "ovl_wilson_tuning": (I, [P, I, ctypes.POINTER(I), DP, DP, DP, DP]),
    "ovl_bench_fp32": (I, [P, DP]),
    "ovl_gram": (I, [P, P, I, P, I, I, I, I, I, I, DP]),
    "ovl_bench_gram": (I, [P, I, I, I, I, I, DP]),
    "ovl_kernel_deflate": (I, [P, I, D, I, I, DP, DP, DP, ctypes.POINTER(I), ctypes.POINTER(I)]),
}


def load():
    """Load liboverlap.so (built by paper_1501_01855_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("liboverlap.so is not built (%s); run paper_1501_01855_gb300.build.build()" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGS.keys())


def _check(status, ctx=None):
    if status != OVL_OK:
        msg = ""
        if ctx:
            msg = load().overlap_last_error(ctx).decode()
        raise OvlError(status, msg)


def _dptr(a):
    return a.ctypes.data_as(DP)


def _spinor_arg(x):
    """(pointer, dtype code, on_device, element count, CUDA device index or None)."""
    try:
        import torch
        if isinstance(x, torch.Tensor):
            if not x.is_contiguous():
                raise ValueError("spinor tensors must be contiguous")
            if x.dtype == torch.complex128:
                code = OVL_C128
            elif x.dtype == torch.complex64:
                code = OVL_C64
            else:
                raise ValueError("spinors must be complex128 or complex64")
            if x.is_cuda:
                return ctypes.c_void_p(x.data_ptr()), code, 1, x.numel(), x.device.index
            if x.requires_grad:
                x = x.detach()
            x = x.numpy()
    except ImportError:
        pass
    x = np.asarray(x)
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("spinor arrays must be C-contiguous")
    if x.dtype == np.complex128:
        code = OVL_C128
    elif x.dtype == np.complex64:
        code = OVL_C64
    else:
        raise ValueError("spinors must be complex128 or complex64")
    return ctypes.c_void_p(x.ctypes.data), code, 0, x.size, None


def _io(ctx_dev, x, out, same_count=True):
    """Marshal an (input, output) pair: both on the same side (host or the context's
    device), the same element type and, unless same_count is False, the same size, so
    that the library never writes past the end of out."""
    pi, code, dev, cnt, di = _spinor_arg(x)
    po, code2, dev2, cnt2, do = _spinor_arg(out)
    if dev != dev2:
        raise ValueError("input and output must both be host arrays or both device tensors")
    if code2 != code:
        raise ValueError("input and output must have the same dtype")
    if same_count and cnt2 != cnt:
        raise ValueError("output holds %d complex entries, input %d" % (cnt2, cnt))
    if dev and ctx_dev is not None and (di != ctx_dev or do != ctx_dev):
        raise ValueError("device tensors must be on cuda:%d, the context's device" % ctx_dev)
    if not dev and isinstance(out, np.ndarray) and not out.flags["WRITEABLE"]:
        raise ValueError("output array is read-only")
    return pi, po, code, dev, cnt


def ovl_version():
    return load().ovl_version().decode()


def ovl_params_default():
    p = ovl_params()
    _check(load().ovl_params_default(ctypes.byref(p)))
    return p


def ovl_zolotarev_coeffs(n, a, b):
    om = np.zeros(n)
    sg = np.zeros(n)
    de = np.zeros(1)
    _check(load().ovl_zolotarev_coeffs(int(n), float(a), float(b), _dptr(om), _dptr(sg), _dptr(de)))
    return om, sg, float(de[0])


def _square_c128(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128))
    if a.ndim != 2 or a.shape[0] != a.shape[1]:
        raise ValueError("expected a square matrix")
    return a


def _cptr(a):
    return a.ctypes.data_as(DP)


def ovl_host_eigh(a):
    """Host Jacobi eigendecomposition of a Hermitian matrix: (w ascending, Z columns)."""
    a = _square_c128(a)
    n = a.shape[0]
    w = np.zeros(n)
    z = np.zeros((n, n), dtype=np.complex128)
    _check(load().ovl_host_eigh(n, _cptr(a), _dptr(w), _cptr(z)))
    return w, z


def ovl_host_cholesky(a):
    """Host Cholesky a = L L^dag (L lower)."""
    a = _square_c128(a)
    l = np.zeros_like(a)
    _check(load().ovl_host_cholesky(a.shape[0], _cptr(a), _cptr(l)))
    return l


def ovl_host_lower_inverse(l):
    l = _square_c128(l)
    li = np.zeros_like(l)
    _check(load().ovl_host_lower_inverse(l.shape[0], _cptr(l), _cptr(li)))
    return li


def ovl_host_lu_solve(a, b):
    """Host pivoted LU solve of a x = b (b: n or n x nb)."""
    a = _square_c128(a)
    b = np.ascontiguousarray(np.asarray(b, dtype=np.complex128))
    vec = b.ndim == 1
    b2 = b.reshape(a.shape[0], -1) if vec else b
    if b2.shape[0] != a.shape[0]:
        raise ValueError("b must have as many rows as a")
    b2 = np.ascontiguousarray(b2)
    x = np.zeros_like(b2)
    _check(load().ovl_host_lu_solve(a.shape[0], _cptr(a), _cptr(b2), b2.shape[1], _cptr(x)))
    return x.ravel() if vec else x


def ovl_host_ritz(E, MVD, G5, mu, delta, keep, restart=False):
    """Host algebra of one Ritz step (Alg. 6) on the k x k Gram blocks of a basis:
    (Ritz values, C (k x kept), residual norms)."""
    E, MVD, G5 = (_square_c128(x) for x in (E, MVD, G5))
    k = E.shape[0]
    if MVD.shape != E.shape or G5.shape != E.shape:
        raise ValueError("E, MVD and G5 must have the same shape")
    ritz, res = np.zeros(2 * keep), np.zeros(2 * keep)
    C = np.zeros((k, 2 * keep), dtype=np.complex128)
    kept = ctypes.c_int()
    _check(load().ovl_host_ritz(k, _cptr(E), _cptr(MVD), _cptr(G5), float(mu), float(delta), int(keep),
                                1 if restart else 0, _dptr(ritz), _cptr(C), _dptr(res), ctypes.byref(kept)))
    n = kept.value
    Cn = C.ravel()[:k * n].reshape(k, n).copy()
    return ritz[:n].copy(), Cn, res[:n].copy()


def ovl_host_sumr_step(rho, dots, state):
    """One step of the library's relSUMR recurrence (host): updates state (11 doubles) in
    place and returns the 9 complex update coefficients."""
    dots = np.ascontiguousarray(np.asarray(dots, dtype=np.float64))
    if dots.size != 4 or state.dtype != np.float64 or state.size != 11 or not state.flags["C_CONTIGUOUS"]:
        raise ValueError("dots: 4 doubles; state: a contiguous float64 array of 11")
    coef = np.zeros(18)
    _check(load().ovl_host_sumr_step(float(rho), _dptr(dots), _dptr(state), _dptr(coef)))
    return coef.view(np.complex128)


def ovl_host_defl_start(VV, WW, WV, G5VV, G5VW, VB, WB, mus, per_vector=False):
    """Host deflated start (Sec. 4) from Gram blocks: the n x nsys coefficients of x0 on psi."""
    VV, WW, WV, G5VV, G5VW = (_square_c128(x) for x in (VV, WW, WV, G5VV, G5VW))
    n = VV.shape[0]
    VB = np.ascontiguousarray(np.asarray(VB, dtype=np.complex128)).reshape(n, -1)
    WB = np.ascontiguousarray(np.asarray(WB, dtype=np.complex128)).reshape(n, -1)
    nsys = VB.shape[1]
    mus = np.ascontiguousarray(np.broadcast_to(np.asarray(mus, dtype=np.float64), (nsys,)))
    if WB.shape != VB.shape or any(x.shape != (n, n) for x in (WW, WV, G5VV, G5VW)):
        raise ValueError("inconsistent Gram block shapes")
    co = np.zeros((n, nsys), dtype=np.complex128)
    _check(load().ovl_host_defl_start(n, _cptr(VV), _cptr(WW), _cptr(WV), _cptr(G5VV), _cptr(G5VW), nsys, _cptr(VB),
                                      _cptr(WB), _dptr(mus), 1 if per_vector else 0, _cptr(co)))
    return co


def ovl_host_rayleigh_ritz(E, H):
    """Rayleigh-Ritz of K from E = X^dag X and H = X^dag K X (host): (theta by |theta|, C)."""
    E, H = _square_c128(E), _square_c128(H)
    m = E.shape[0]
    th = np.zeros(m)
    C = np.zeros((m, m), dtype=np.complex128)
    _check(load().ovl_host_rayleigh_ritz(m, _cptr(E), _cptr(H), _dptr(th), _cptr(C)))
    return th, C


def ovl_host_tridiag_extremes(d, e):
    """Smallest and largest eigenvalue of the symmetric tridiagonal (d, e)."""
    d = np.ascontiguousarray(np.asarray(d, dtype=np.float64))
    e = np.ascontiguousarray(np.asarray(e, dtype=np.float64))
    if e.size != max(0, d.size - 1):
        raise ValueError("e must hold len(d) - 1 entries")
    lo, hi = np.zeros(1), np.zeros(1)
    ep = _dptr(e) if e.size else None
    _check(load().ovl_host_tridiag_extremes(d.size, _dptr(d), ep, _dptr(lo), _dptr(hi)))
    return float(lo[0]), float(hi[0])


def _current_device():
    try:
        import torch
        return torch.cuda.current_device() if torch.cuda.is_available() else None
    except ImportError:
        return None


def links_digest(links):
    """Digest of a gauge field in the canonical complex128 layout (bytes as given)."""
    import hashlib
    a = np.ascontiguousarray(np.asarray(links, dtype=np.complex128))
    return hashlib.blake2b(a.view(np.uint8), digest_size=16).hexdigest()


class Overlap:
    """One overlap context (gauge field, m0, default mu, Zolotarev order)."""

    def __init__(self, dims, links, m0, mu, n_poles, eps_sign, params=None, **kw):
        lib = load()
        if params is None:
            params = ovl_params_default()
        for k, v in kw.items():
            setattr(params, k, v)
        self.params = params
        self.dims = tuple(int(d) for d in dims)
        self.V = int(np.prod(self.dims))
        links = np.ascontiguousarray(np.asarray(links, dtype=np.complex128))
        if links.size != self.V * 36:
            raise ValueError("links must hold 4*9*V complex entries")
        d4 = (ctypes.c_int * 4)(*self.dims)
        h = ctypes.c_void_p()
        st = lib.overlap_create(ctypes.byref(h), d4, links.ctypes.data_as(DP), float(m0), float(mu), int(n_poles),
                                float(eps_sign), ctypes.byref(params))
        if st != OVL_OK:
            raise OvlError(st, "overlap_create failed (see stderr)")
        self.h = h
        self.m0, self.mu, self.n_poles = m0, mu, n_poles
        self.device = _current_device()
        # fingerprint of the gauge field the library copied (checked by the autograd wrapper)
        self.links_digest = links_digest(links)

    def trim(self):
        """Release the workspaces and graphs the context caches between calls."""
        _check(load().ovl_trim(self.h), self.h)

    def close(self):
        if getattr(self, "h", None):
            load().overlap_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _n(self, count):
        n, r = divmod(count, self.V * 12)
        if r or n < 1:
            raise ValueError("spinor buffer size is not a multiple of 12*V")
        return n

    def zolotarev(self):
        om = np.zeros(64)
        sg = np.zeros(64)
        de, a, b = np.zeros(1), np.zeros(1), np.zeros(1)
        _check(load().overlap_zolotarev(self.h, _dptr(om), _dptr(sg), _dptr(de), _dptr(a), _dptr(b)), self.h)
        return om[:self.n_poles].copy(), sg[:self.n_poles].copy(), float(de[0]), float(a[0]), float(b[0])

    def kernel_deflate(self, n_ev, tol=1e-10, max_iter=100, n_poles=0):
        """Deflate the n_ev lowest-|lambda| eigenvectors of K from the sign function and
        narrow the rational to the rest of the spectrum (n_ev = 0 undoes it). Returns
        (lambda, residuals, a', poles in use, filter steps)."""
        lam = np.zeros(max(n_ev, 1))
        res = np.zeros(max(n_ev, 1))
        a = ctypes.c_double()
        npu, its = ctypes.c_int(), ctypes.c_int()
        _check(load().ovl_kernel_deflate(self.h, int(n_ev), float(tol), int(max_iter), int(n_poles), _dptr(lam),
                                         _dptr(res), ctypes.byref(a), ctypes.byref(npu), ctypes.byref(its)), self.h)
        self.n_poles = npu.value
        return lam[:n_ev].copy(), res[:n_ev].copy(), a.value, npu.value, its.value

    def wilson_apply(self, x, out, prec=OVL_PREC_F64):
        pi, po, code, dev, cnt = _io(self.device, x, out)
        _check(load().ovl_wilson_apply(self.h, pi, po, self._n(cnt), code, dev, int(prec)), self.h)
        return out

    def wilson_apply_noalloc(self, x, out, prec=OVL_PREC_F64):
        """K on device tensors without any allocation during the call (static scratch)."""
        pi, po, code, dev, cnt = _io(self.device, x, out)
        if not dev:
            raise ValueError("ovl_wilson_apply_noalloc takes device buffers only")
        _check(load().ovl_wilson_apply_noalloc(self.h, pi, po, self._n(cnt), code, int(prec)), self.h)
        return out

    def sign_apply(self, x, out, eta=0.0, prec=OVL_PREC_AUTO):
        pi, po, code, dev, cnt = _io(self.device, x, out)
        _check(load().ovl_sign_apply(self.h, pi, po, self._n(cnt), code, dev, float(eta), int(prec)), self.h)
        return out

    def apply(self, x, out, mu=None, eta=0.0, prec=OVL_PREC_AUTO, hermitian=False):
        pi, po, code, dev, cnt = _io(self.device, x, out)
        mu = self.mu if mu is None else mu
        _check(load().overlap_apply(self.h, float(mu), pi, po, self._n(cnt), code, dev, float(eta), int(prec),
                                    1 if hermitian else 0), self.h)
        return out

    def sumr(self, b, x, tol, eta_fixed=0.0, maxit=200, mu=None):
        pb, px, code, dev, cnt = _io(self.device, b, x)
        n = self._n(cnt)
        mu = self.mu if mu is None else mu
        hist = np.zeros(n * maxit)
        its = (ctypes.c_int * n)()
        _check(load().overlap_sumr(self.h, float(mu), pb, px, n, code, dev, float(tol), float(eta_fixed), int(maxit),
                                   _dptr(hist), its), self.h)
        its = list(its)
        return [hist[j * maxit:j * maxit + its[j]] for j in range(n)], its

    def solve(self, b, x, tol, mus=None, defl=None, allow_noconv=False):
        pb, px, code, dev, cnt = _io(self.device, b, x, same_count=False)
        nrhs = self._n(cnt)
        mus = np.ascontiguousarray([self.mu] if mus is None else mus, dtype=np.float64)
        if _spinor_arg(x)[3] != cnt * len(mus):
            raise ValueError("x must hold nmass * nrhs spinors")
        info = (ovl_solve_info * (nrhs * len(mus)))()
        st = load().overlap_solve(self.h, nrhs, _dptr(mus), len(mus), pb, px, code, dev, float(tol),
                                  defl.h if defl is not None else None, info)
        if not (st == OVL_OK or (allow_noconv and st == OVL_ENOCONV)):
            _check(st, self.h)
        return [i.as_dict() for i in info]

    def eigsumr_accumulate(self, b, x, tol, n_eig, m_basis, mu=None, defl=None, allow_noconv=False):
        pb, px, code, dev, cnt = _io(self.device, b, x)
        if self._n(cnt) != 1:
            raise ValueError("eigsumr_accumulate takes one source")
        mu = self.mu if mu is None else mu
        h = ctypes.c_void_p(defl.h.value if defl is not None else None)
        info = (ovl_solve_info * 1)()
        st = load().eigsumr_accumulate(self.h, ctypes.byref(h), int(n_eig), int(m_basis), float(mu), pb, px, code,
                                       dev, float(tol), info)
        if st not in (OVL_OK, OVL_ENOCONV):
            _check(st, self.h)
        if defl is None:
            defl = Deflation(self, h)
        if st == OVL_ENOCONV and not allow_noconv:
            # the space is kept (and refined) even when the solve itself fell short
            raise OvlError(st, load().overlap_last_error(self.h).decode())
        return defl, info[0].as_dict()

    def force(self, phi, mu=None, tol=1e-10):
        pp, code, dev, cnt, di = _spinor_arg(phi)
        if self._n(cnt) != 1:
            raise ValueError("overlap_force takes one source phi")
        if dev and self.device is not None and di != self.device:
            raise ValueError("phi must be on cuda:%d, the context's device" % self.device)
        mu = self.mu if mu is None else mu
        G = np.zeros(self.V * 36 * 2)
        S = np.zeros(1)
        _check(load().overlap_force(self.h, float(mu), pp, code, dev, float(tol), _dptr(G), _dptr(S)), self.h)
        Gc = G.view(np.complex128).reshape(tuple(reversed(self.dims)) + (4, 3, 3))
        return Gc, float(S[0])

    def eigensolve(self, n_eig, m_basis, max_steps, res_tol=0.0, mu=None, start=None, defl=None, round_diags=24):
        """Standalone eigSUMR eigensolver (ovl_eigensolve): returns (space, steps used)."""
        mu = self.mu if mu is None else mu
        if start is not None:
            ps, code, dev, cnt, ds = _spinor_arg(start)
            if self._n(cnt) != 1:
                raise ValueError("start must be one spinor")
            if dev and self.device is not None and ds != self.device:
                raise ValueError("start must be on cuda:%d, the context's device" % self.device)
        else:
            ps, code, dev = None, OVL_C128, 0
        h = ctypes.c_void_p(defl.h.value if defl is not None else None)
        used = ctypes.c_int()
        _check(load().ovl_eigensolve(self.h, ctypes.byref(h), int(n_eig), int(m_basis), float(mu), ps, code, dev,
                                     int(max_steps), float(res_tol), int(round_diags), ctypes.byref(used)), self.h)
        if defl is None:
            defl = Deflation(self, h)
        return defl, used.value

    def ritz_recalculate(self, v, vD, n_keep, mu=None, delta=0.01):
        """Alg. 6 on the basis v (m spinors) with v^D = D(mu) v: (Ritz values, new v,
        new v^D, residuals) of the lowest n_keep Ritz pairs."""
        pv, pd, code, dev, cnt = _io(self.device, v, vD)
        m = self._n(cnt)
        mu = self.mu if mu is None else mu
        if dev:
            import torch
            vo = torch.empty((n_keep,) + tuple(v.shape[1:]), dtype=v.dtype, device=v.device)
            vdo = torch.empty_like(vo)
        else:
            vo = np.empty((n_keep,) + tuple(np.shape(v)[1:]), dtype=np.asarray(v).dtype)
            vdo = np.empty_like(vo)
        ritz = np.zeros(n_keep)
        res = np.zeros(n_keep)
        _check(load().ovl_ritz_recalculate(self.h, m, int(n_keep), float(mu), float(delta), pv, pd,
                                           _spinor_arg(vo)[0], _spinor_arg(vdo)[0], code, dev, _dptr(ritz),
                                           _dptr(res)), self.h)
        return ritz, vo, vdo, res

    def profile_enable(self, on=True):
        _check(load().ovl_profile_enable(self.h, 1 if on else 0), self.h)

    def profile_reset(self):
        _check(load().ovl_profile_reset(self.h), self.h)

    def profile_get(self):
        out = {}
        for c in range(OVL_PROF_CLASSES):
            n = ctypes.c_longlong()
            ms, by = ctypes.c_double(), ctypes.c_double()
            _check(load().ovl_profile_get(self.h, c, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by)), self.h)
            u = ctypes.c_double()
            _check(load().ovl_profile_units(self.h, c, ctypes.byref(u)), self.h)
            out[PROF_NAMES[c]] = {"launches": n.value, "ms": ms.value, "bytes": by.value, "units": u.value}
        return out

    def wilson_tuning(self, prec):
        """(variant in use, ms per launch of variants 0, 1, 2, 3) from the create-time autotuner."""
        v = ctypes.c_int()
        t = [ctypes.c_double() for _ in range(4)]
        _check(load().ovl_wilson_tuning(self.h, int(prec), ctypes.byref(v), *[ctypes.byref(x) for x in t]), self.h)
        return (v.value,) + tuple(x.value for x in t)

    def bench_fp32(self):
        """Measured FP32 FMA instructions per second of the context's device."""
        r = ctypes.c_double()
        _check(load().ovl_bench_fp32(self.h, ctypes.byref(r)), self.h)
        return r.value

    def gram(self, A, B, g5=0, prec=OVL_PREC_F64, method=0):
        """G[i, j] = (A_i, [gamma5] B_j) for spinor batches A (na) and B (nb), same dtype
        and device; returns an na x nb complex128 NumPy array."""
        pa, code, dev, cnta, da = _spinor_arg(A)
        pb, codeb, devb, cntb, db = _spinor_arg(B)
        if code != codeb or dev != devb or (dev and da != db):
            raise ValueError("A and B must share dtype and device")
        if dev and self.device is not None and da != self.device:
            raise ValueError("A and B must be on cuda:%d, the context's device" % self.device)
        na, nb = self._n(cnta), self._n(cntb)
        G = np.zeros(na * nb * 2)
        _check(load().ovl_gram(self.h, pa, na, pb, nb, code, dev, int(prec), int(g5), int(method), _dptr(G)), self.h)
        return G.view(np.complex128).reshape(na, nb)

    def bench_gram(self, prec, na, nb, method=0, iters=3):
        """Mean milliseconds of one na x nb Gram block on library-held random fields."""
        ms = ctypes.c_double()
        _check(load().ovl_bench_gram(self.h, int(prec), int(na), int(nb), int(method), int(iters),
                                     ctypes.byref(ms)), self.h)
        return ms.value

    def bench_wilson(self, prec, n, iters):
        ms, by = ctypes.c_double(), ctypes.c_double()
        _check(load().ovl_bench_wilson(self.h, int(prec), int(n), int(iters), ctypes.byref(ms), ctypes.byref(by)),
               self.h)
        return ms.value, by.value


class Deflation:
    """A deflation space from eigsumr_accumulate (or ovl_defl_load)."""

    def __init__(self, ctx, handle):
        self.ctx = ctx
        self.h = handle

    def info(self):
        n = ctypes.c_int()
        _check(load().ovl_defl_info(self.h, ctypes.byref(n), None, None))
        r = np.zeros(max(1, n.value))
        s = np.zeros(max(1, n.value))
        _check(load().ovl_defl_info(self.h, ctypes.byref(n), _dptr(r), _dptr(s)))
        return r[:n.value], s[:n.value]

    def vector(self, i):
        v = np.zeros(self.ctx.V * 12, dtype=np.complex128)
        vd = np.zeros(self.ctx.V * 12, dtype=np.complex128)
        _check(load().ovl_defl_vector(self.h, int(i), v.view(np.float64).ctypes.data_as(DP),
                                      vd.view(np.float64).ctypes.data_as(DP)))
        shp = tuple(reversed(self.ctx.dims)) + (4, 3)
        return v.reshape(shp), vd.reshape(shp)

    def save(self, path):
        _check(load().ovl_defl_save(self.h, path.encode()))

    @classmethod
    def load_file(cls, ctx, path):
        h = ctypes.c_void_p()
        _check(load().ovl_defl_load(ctx.h, ctypes.byref(h), path.encode()), ctx.h)
        return cls(ctx, h)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            load().ovl_defl_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
