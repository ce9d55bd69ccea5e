"""Python binding of libwt, the GB300 (sm_103a) CUDA library for the
hybrid-spectral free-surface Navier-Stokes wave tank (C ABI: include/wt.h).

Only argument marshalling happens here: every step of the computation runs in
the CUDA kernels of ``csrc/``.  Arrays may be numpy float64 arrays (host
memory) or contiguous float64 torch CUDA tensors (device memory); the library
detects which.  Importing fails loudly when libwt.so has not been built
(``paper_2406_00991_gb300.build.build()``); there is no CPU fallback.

The functions keep the C names (``wt_create``, ``wt_poisson_solve``,
``wt_rk_stage``, ``wt_step`` ...) and return the status code; ``Tank`` wraps
them and raises ``WtError`` on a non-zero status.
"""

import ctypes
import os

import numpy as np

from .build import LIB as _LIB_PATH

WT_OK, WT_EINVAL, WT_ENOMEM, WT_ENOCONV, WT_EBREAK, WT_ECUDA, WT_ETIMEOUT, WT_ENOTSUP = range(8)
WT_FP64, WT_MIXED, WT_FP32, WT_REFINE = 0, 1, 2, 3
STATUS_NAMES = {0: "WT_OK", 1: "WT_EINVAL", 2: "WT_ENOMEM", 3: "WT_ENOCONV", 4: "WT_EBREAK",
                5: "WT_ECUDA", 6: "WT_ETIMEOUT", 7: "WT_ENOTSUP"}


class wt_options(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("tol", ctypes.c_double), ("restart", ctypes.c_int),
                ("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("omega", ctypes.c_double),
                ("max_it", ctypes.c_int),
                ("filter", ctypes.c_int), ("linear", ctypes.c_int), ("coarsest_max", ctypes.c_int),
                ("bc_transfer", ctypes.c_int), ("tail_max", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("max_ir", ctypes.c_int), ("vcycle_grid", ctypes.c_int),
                ("tail_cluster", ctypes.c_int), ("barrier_cycles", ctypes.c_longlong),
                ("cycle", ctypes.c_int), ("smoother", ctypes.c_int), ("omega_s", ctypes.c_double),
                ("warp_fft", ctypes.c_int),
                ("pdl", ctypes.c_int),
                ("df64", ctypes.c_int),
                ("spectral_min", ctypes.c_int)]


class wt_solve_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("status", ctypes.c_int), ("refinements", ctypes.c_int)]


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError("libwt.so is not built (run paper_2406_00991_gb300.build.build()); "
                          "this package has no CPU fallback")
    lib = ctypes.CDLL(_LIB_PATH)
    P = ctypes.c_void_p
    D = ctypes.c_double
    I = ctypes.c_int
    sig = {
        "wt_default_options": [ctypes.POINTER(wt_options)],
        "wt_create": [I, I, I, D, D, D, P, ctypes.POINTER(P)],
        "wt_set_options": [P, ctypes.POINTER(wt_options)],
        "wt_get_options": [P, ctypes.POINTER(wt_options)],
        "wt_set_stream": [P, P],
        "wt_get_grid": [P, P, P, P],
        "wt_get_levels": [P, ctypes.POINTER(I), P],
        "wt_levels_for": [I, I, I, I, ctypes.POINTER(I), P],
        "wt_sigma_matrices": [I, I, I, P, P, P, P],
        "wt_set_state": [P, P, P, P, P, D],
        "wt_get_state": [P, P, P, P, P, ctypes.POINTER(D)],
        "wt_get_pressure": [P, P],
        "wt_apply_operator": [P, P, P, P, P, I],
        "wt_precondition": [P, P, P, P, P, I],
        "wt_poisson_solve": [P, P, P, P, P, D, ctypes.POINTER(wt_solve_info)],
        "wt_rk_stage": [P, I, D],
        "wt_step": [P, D, I],
        "wt_get_stats": [P, ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_long)],
        "wt_destroy": [P],
        "wt_profile": [P, ctypes.c_uint],
        "wt_profile_read": [P, I, ctypes.POINTER(D), ctypes.POINTER(ctypes.c_long),
                            ctypes.POINTER(D), ctypes.POINTER(D)],
        "wt_get_launches": [P, ctypes.POINTER(ctypes.c_long)],
        "wt_apply_operator_static": [I, I, D, P, P, P, P, P, P],
        "wt_autotune": [P, P, P, P, I, ctypes.POINTER(wt_options), ctypes.POINTER(D), ctypes.POINTER(D)],
        "wt_autotune_step": [P, D, I, ctypes.POINTER(wt_options), ctypes.POINTER(D), ctypes.POINTER(D)],
        "wt_autotune_cache": [ctypes.c_char_p],
        "wt_set_bathymetry": [P, P],
        "wt_apply_operator_transposed": [P, P, P, P, P, I],
        "wt_adjoint_solve": [P, P, P, P, P, D, ctypes.POINTER(wt_solve_info)],
        "wt_adjoint_step": [P, D, P, P, P, P, P, P, P],
        "wt_create_batch": [I, P, P, P, D, D, P, ctypes.POINTER(P)],
        "wt_batch_set_options": [P, ctypes.POINTER(wt_options)],
        "wt_batch_set_state": [P, I, P, P, P, D],
        "wt_batch_get_state": [P, I, P, P, P, ctypes.POINTER(D)],
        "wt_batch_step": [P, P, I],
        "wt_batch_stats": [P, I, ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_long),
                           ctypes.POINTER(D)],
        "wt_batch_destroy": [P],
        "wt_batch_set_stream": [P, P],
        "wt_batch_size": [P, ctypes.POINTER(I)],
        "wt_batch_tank_dims": [P, I, ctypes.POINTER(I), ctypes.POINTER(I)],
        "wt_batch_get_options": [P, ctypes.POINTER(wt_options)],
        "wt_batch_autotune": [P, P, I, ctypes.POINTER(wt_options), ctypes.POINTER(D), ctypes.POINTER(D)],
        "wt_time_kernel": [P, P, P, I, I, I, ctypes.POINTER(D), ctypes.POINTER(ctypes.c_long)],
        "wt_stream_function_wave": [P, I, D, I, D, P, P, P, ctypes.POINTER(D)],
        "wt_stream_function_solve": [D, D, D, D, I, P, P, P],
        "wt_relax": [P, D, D, P, P, P, P],
        "wt_last_error": [ctypes.c_char_p, ctypes.c_size_t],
    }
    for name, args in sig.items():
        try:
            f = getattr(lib, name)
        except AttributeError as e:
            raise ImportError("libwt.so is stale (missing %s): rebuild it" % name) from e
        f.argtypes = args
        f.restype = I
    return lib


class _Lazy:
    """The library, loaded at its first use: importing the package (for
    instance to build the library) loads nothing, so a build in the same
    process is what the first call sees.  A missing or stale libwt.so raises
    ImportError at that first call; there is no CPU fallback."""

    def __init__(self):
        self._real = None

    def __getattr__(self, name):
        if self._real is None:
            self._real = _load()
        return getattr(self._real, name)


def _reload():
    """Load libwt.so (after a build); returns the ctypes library."""
    global _lib, lib
    _lib = _load()
    lib = _lib
    return _lib


_lib = _Lazy()
lib = _lib


def _ptr(a):
    """Device pointer of a float64 CUDA tensor or host pointer of a float64 numpy array."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if a.dtype.__repr__() != "torch.float64" or not a.is_contiguous():
            raise TypeError("torch tensors passed to libwt must be contiguous float64")
        return ctypes.c_void_p(a.data_ptr())
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]):
        raise TypeError("numpy arrays passed to libwt must be C-contiguous float64")
    return a.ctypes.data_as(ctypes.c_void_p)


def wt_last_error():
    buf = ctypes.create_string_buffer(512)
    code = _lib.wt_last_error(buf, 512)
    return code, buf.value.decode()


def wt_default_options():
    o = wt_options()
    _lib.wt_default_options(ctypes.byref(o))
    return o


def wt_create(Nx, Ny, Nz, L, g, nu, bathymetry):
    h = ctypes.c_void_p()
    st = _lib.wt_create(int(Nx), int(Ny), int(Nz), float(L), float(g), float(nu), _ptr(bathymetry),
                        ctypes.byref(h))
    return st, h


def wt_set_options(t, opt):
    return _lib.wt_set_options(t, ctypes.byref(opt))


def wt_get_options(t):
    o = wt_options()
    st = _lib.wt_get_options(t, ctypes.byref(o))
    return st, o


def wt_set_stream(t, stream_handle):
    return _lib.wt_set_stream(t, ctypes.c_void_p(int(stream_handle)))


def wt_get_grid(t, x, y, sigma):
    return _lib.wt_get_grid(t, _ptr(x), _ptr(y), _ptr(sigma))


def wt_get_levels(t):
    n = ctypes.c_int()
    dims = (ctypes.c_int * 48)()
    st = _lib.wt_get_levels(t, ctypes.byref(n), dims)
    return st, [tuple(dims[3 * l: 3 * l + 3]) for l in range(n.value)]


def wt_levels_for(Nx, Ny, Nz, coarsest_max):
    """Host only: the level sizes wt_create would build (no tank, no GPU)."""
    n = ctypes.c_int()
    dims = (ctypes.c_int * 48)()
    st = _lib.wt_levels_for(int(Nx), int(Ny), int(Nz), int(coarsest_max), ctypes.byref(n), dims)
    return st, [tuple(dims[3 * l: 3 * l + 3]) for l in range(n.value)]


def wt_sigma_matrices(Nz, Nzc, bc_transfer=0):
    """Host only: (status, D, F, R, P), the library's sigma-direction
    derivative, filter, restriction and prolongation matrices (no GPU)."""
    M1, Mc = max(int(Nz) + 1, 1), max(int(Nzc) + 1, 1)     # sizes the library rejects write nothing
    D, F = np.zeros((M1, M1)), np.zeros((M1, M1))
    R, Pm = np.zeros((Mc, M1)), np.zeros((M1, Mc))
    st = _lib.wt_sigma_matrices(int(Nz), int(Nzc), int(bc_transfer), D.ctypes.data, F.ctypes.data,
                                R.ctypes.data, Pm.ctypes.data)
    return st, D, F, R, Pm


def wt_set_state(t, eta, u, v, w, time=0.0):
    return _lib.wt_set_state(t, _ptr(eta), _ptr(u), _ptr(v), _ptr(w), float(time))


def wt_get_state(t, eta, u, v, w):
    tm = ctypes.c_double()
    st = _lib.wt_get_state(t, _ptr(eta), _ptr(u), _ptr(v), _ptr(w), ctypes.byref(tm))
    return st, tm.value


def wt_get_pressure(t, p):
    return _lib.wt_get_pressure(t, _ptr(p))


def wt_apply_operator(t, eta_a, eta_b, p, Ap, precision=WT_FP64):
    return _lib.wt_apply_operator(t, _ptr(eta_a), _ptr(eta_b), _ptr(p), _ptr(Ap), int(precision))


def wt_precondition(t, eta_a, eta_b, r, z, precision=WT_FP64):
    return _lib.wt_precondition(t, _ptr(eta_a), _ptr(eta_b), _ptr(r), _ptr(z), int(precision))


def wt_poisson_solve(t, eta_a, eta_b, rhs, p, tol=0.0):
    info = wt_solve_info()
    st = _lib.wt_poisson_solve(t, _ptr(eta_a), _ptr(eta_b), _ptr(rhs), _ptr(p), float(tol),
                               ctypes.byref(info))
    return st, info


def wt_rk_stage(t, k, dt):
    return _lib.wt_rk_stage(t, int(k), float(dt))


def wt_step(t, dt, nsteps):
    return _lib.wt_step(t, float(dt), int(nsteps))


def wt_get_stats(t):
    s, i = ctypes.c_long(), ctypes.c_long()
    st = _lib.wt_get_stats(t, ctypes.byref(s), ctypes.byref(i))
    return st, s.value, i.value


def wt_destroy(t):
    return _lib.wt_destroy(t)


KERNEL_CLASSES = ["rowpass", "opcols", "smooth", "colmat", "blockinv", "coarse", "krylov", "stage",
                  "tail"]


def wt_profile(t, mask):
    return _lib.wt_profile(t, ctypes.c_uint(mask))


def wt_profile_read(t, kernel_class):
    ms, b, f = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    n = ctypes.c_long()
    st = _lib.wt_profile_read(t, int(kernel_class), ctypes.byref(ms), ctypes.byref(n), ctypes.byref(b),
                              ctypes.byref(f))
    return st, ms.value, n.value, b.value, f.value


def wt_apply_operator_static(Nx, Nz, L, h, eta_a, eta_b, p, Ap, stream_handle=0):
    """Allocation-free 2D FP64 operator apply; every array must be a CUDA tensor."""
    return _lib.wt_apply_operator_static(int(Nx), int(Nz), float(L), _ptr(h), _ptr(eta_a), _ptr(eta_b),
                                         _ptr(p), _ptr(Ap), ctypes.c_void_p(int(stream_handle)))


def wt_stream_function_wave(t, nwaves, H, nmodes, time, eta, u, w):
    c = ctypes.c_double()
    st = _lib.wt_stream_function_wave(t, int(nwaves), float(H), int(nmodes), float(time), _ptr(eta), _ptr(u),
                                      _ptr(w), ctypes.byref(c))
    return st, c.value


def wt_stream_function_solve(k, d, H, g, nmodes):
    """Host only: (status, (c, Q, R), B[nmodes], E[nmodes + 1]) of the
    stream-function wave (no tank, no GPU)."""
    params = np.zeros(3)
    B = np.zeros(int(nmodes))
    E = np.zeros(int(nmodes) + 1)
    st = _lib.wt_stream_function_solve(float(k), float(d), float(H), float(g), int(nmodes),
                                       params.ctypes.data, B.ctypes.data, E.ctypes.data)
    return st, tuple(params), B, E


def wt_relax(t, x0, x1, eta_target, u_target, v_target, w_target):
    return _lib.wt_relax(t, float(x0), float(x1), _ptr(eta_target), _ptr(u_target), _ptr(v_target),
                         _ptr(w_target))


WT_TIME_OPERATOR, WT_TIME_VCYCLE = 0, 1


def wt_time_kernel(t, eta_a, eta_b, what, precision, reps):
    ms, n = ctypes.c_double(), ctypes.c_long()
    st = _lib.wt_time_kernel(t, _ptr(eta_a), _ptr(eta_b), int(what), int(precision), int(reps),
                             ctypes.byref(ms), ctypes.byref(n))
    return st, ms.value, n.value


def wt_set_bathymetry(t, h):
    return _lib.wt_set_bathymetry(t, _ptr(h))


def wt_apply_operator_transposed(t, eta_a, eta_b, lam, out, precision=WT_FP64):
    return _lib.wt_apply_operator_transposed(t, _ptr(eta_a), _ptr(eta_b), _ptr(lam), _ptr(out), int(precision))


def wt_adjoint_solve(t, eta_a, eta_b, rhs, lam, tol=0.0):
    info = wt_solve_info()
    st = _lib.wt_adjoint_solve(t, _ptr(eta_a), _ptr(eta_b), _ptr(rhs), _ptr(lam), float(tol),
                               ctypes.byref(info))
    return st, info


def wt_adjoint_step(t, dt, eta, u, w, lam_eta, lam_u, lam_w, dJ_dh=None):
    return _lib.wt_adjoint_step(t, float(dt), _ptr(eta), _ptr(u), _ptr(w), _ptr(lam_eta), _ptr(lam_u),
                                _ptr(lam_w), _ptr(dJ_dh))


def wt_autotune(t, eta_a, eta_b, rhs, reps=3):
    o = wt_options()
    b, e = ctypes.c_double(), ctypes.c_double()
    st = _lib.wt_autotune(t, _ptr(eta_a), _ptr(eta_b), _ptr(rhs), int(reps), ctypes.byref(o),
                          ctypes.byref(b), ctypes.byref(e))
    return st, o, b.value, e.value


def wt_autotune_step(t, dt, reps=3):
    o = wt_options()
    b, e = ctypes.c_double(), ctypes.c_double()
    st = _lib.wt_autotune_step(t, float(dt), int(reps), ctypes.byref(o), ctypes.byref(b), ctypes.byref(e))
    return st, o, b.value, e.value


def wt_autotune_cache(path):
    """File of tuned options for wt_autotune / wt_autotune_step (None: none)."""
    return _lib.wt_autotune_cache(None if path is None else os.fsencode(path))


def wt_create_batch(Nx, Nz, L, bathymetry, g=9.81, nu=0.0):
    """Batch of 2D tanks; bathymetry is a list of float64 arrays (host or device)."""
    n = len(Nx)
    nx = np.ascontiguousarray(Nx, dtype=np.int32)
    nz = np.ascontiguousarray(Nz, dtype=np.int32)
    ll = np.ascontiguousarray(L, dtype=np.float64)
    hp = (ctypes.c_void_p * n)(*[_ptr(h).value for h in bathymetry])
    b = ctypes.c_void_p()
    st = _lib.wt_create_batch(n, nx.ctypes.data_as(ctypes.c_void_p), nz.ctypes.data_as(ctypes.c_void_p),
                              ll.ctypes.data_as(ctypes.c_void_p), g, nu, ctypes.cast(hp, ctypes.c_void_p),
                              ctypes.byref(b))
    return st, b


def wt_batch_set_options(b, o):
    return _lib.wt_batch_set_options(b, ctypes.byref(o))


def wt_batch_set_state(b, i, eta, u, w, time=0.0):
    return _lib.wt_batch_set_state(b, int(i), _ptr(eta), _ptr(u), _ptr(w), float(time))


def wt_batch_get_state(b, i, eta, u, w):
    tm = ctypes.c_double()
    st = _lib.wt_batch_get_state(b, int(i), _ptr(eta), _ptr(u), _ptr(w), ctypes.byref(tm))
    return st, tm.value


def wt_batch_step(b, dt, nsteps):
    d = np.ascontiguousarray(dt, dtype=np.float64)
    return _lib.wt_batch_step(b, d.ctypes.data_as(ctypes.c_void_p), int(nsteps))


def wt_batch_stats(b, i):
    s, it, r = ctypes.c_long(), ctypes.c_long(), ctypes.c_double()
    st = _lib.wt_batch_stats(b, int(i), ctypes.byref(s), ctypes.byref(it), ctypes.byref(r))
    return st, s.value, it.value, r.value


def wt_batch_destroy(b):
    return _lib.wt_batch_destroy(b)


def wt_batch_set_stream(b, stream_handle):
    return _lib.wt_batch_set_stream(b, ctypes.c_void_p(int(stream_handle)))


def wt_batch_size(b):
    n = ctypes.c_int()
    st = _lib.wt_batch_size(b, ctypes.byref(n))
    return st, n.value


def wt_batch_tank_dims(b, i):
    nx, nz = ctypes.c_int(), ctypes.c_int()
    st = _lib.wt_batch_tank_dims(b, int(i), ctypes.byref(nx), ctypes.byref(nz))
    return st, nx.value, nz.value


def wt_batch_get_options(b):
    o = wt_options()
    st = _lib.wt_batch_get_options(b, ctypes.byref(o))
    return st, o


def wt_batch_autotune(b, dt, reps=1):
    d = np.ascontiguousarray(dt, dtype=np.float64)
    o = wt_options()
    bm, em = ctypes.c_double(), ctypes.c_double()
    st = _lib.wt_batch_autotune(b, d.ctypes.data_as(ctypes.c_void_p), int(reps), ctypes.byref(o),
                                ctypes.byref(bm), ctypes.byref(em))
    return st, o, bm.value, em.value


def wt_get_launches(t):
    n = ctypes.c_long()
    st = _lib.wt_get_launches(t, ctypes.byref(n))
    return st, n.value


class WtError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(code, code), msg))
        self.code = code


def _check(st):
    if st != WT_OK:
        code, msg = wt_last_error()
        raise WtError(st, msg)


class Tank:
    """Owning wrapper of a wt_tank handle; methods raise WtError on failure."""

    def __init__(self, Nx, Ny, Nz, L, bathymetry, g=9.81, nu=0.0, **options):
        self.Nx, self.Ny, self.Nz, self.L = int(Nx), int(Ny), int(Nz), float(L)
        self.M1 = self.Nz + 1
        st, h = wt_create(Nx, Ny, Nz, L, g, nu, np.ascontiguousarray(bathymetry, dtype=np.float64)
                          if not hasattr(bathymetry, "data_ptr") else bathymetry)
        _check(st)
        self.handle = h
        if options:
            self.set_options(**options)

    @property
    def shape(self):
        return (self.M1, self.Ny, self.Nx)

    def options(self):
        st, o = wt_get_options(self.handle)
        _check(st)
        return {k: getattr(o, k) for k, _ in wt_options._fields_}

    def set_options(self, **kw):
        st, o = wt_get_options(self.handle)
        _check(st)
        for k, v in kw.items():
            if k not in dict(wt_options._fields_):
                raise KeyError(k)
            setattr(o, k, v)
        _check(wt_set_options(self.handle, o))

    def set_stream(self, stream_handle):
        _check(wt_set_stream(self.handle, stream_handle))

    def grid(self):
        x = np.zeros(self.Nx)
        y = np.zeros(self.Ny)
        s = np.zeros(self.M1)
        _check(wt_get_grid(self.handle, x, y, s))
        return x, y, s

    def levels(self):
        st, lv = wt_get_levels(self.handle)
        _check(st)
        return lv

    def set_state(self, eta, u, v, w, time=0.0):
        _check(wt_set_state(self.handle, eta, u, v, w, time))

    def get_state(self):
        eta = np.zeros((self.Ny, self.Nx))
        u, v, w = (np.zeros(self.shape) for _ in range(3))
        st, tm = wt_get_state(self.handle, eta, u, v, w)
        _check(st)
        return eta, u, v, w, tm

    def pressure(self):
        p = np.zeros(self.shape)
        _check(wt_get_pressure(self.handle, p))
        return p

    def apply_operator(self, eta_a, eta_b, p, precision=WT_FP64, out=None):
        out = np.zeros(self.shape) if out is None else out
        _check(wt_apply_operator(self.handle, eta_a, eta_b, p, out, precision))
        return out

    def precondition(self, eta_a, eta_b, r, precision=WT_FP64, out=None):
        out = np.zeros(self.shape) if out is None else out
        _check(wt_precondition(self.handle, eta_a, eta_b, r, out, precision))
        return out

    def poisson_solve(self, eta_a, eta_b, rhs, p=None, tol=0.0, raise_noconv=True):
        p = np.zeros(self.shape) if p is None else p
        st, info = wt_poisson_solve(self.handle, eta_a, eta_b, rhs, p, tol)
        if st != WT_OK and (st != WT_ENOCONV or raise_noconv):
            _check(st)
        return p, info

    def rk_stage(self, k, dt):
        _check(wt_rk_stage(self.handle, k, dt))

    def autotune_step(self, dt, reps=3):
        """Pick the fastest settings for one step from the current state (restored)."""
        st, o, best, entry = wt_autotune_step(self.handle, dt, reps)
        _check(st)
        return {k: getattr(o, k) for k, _ in wt_options._fields_}, best, entry

    def set_bathymetry(self, h):
        _check(wt_set_bathymetry(self.handle, h))

    def apply_operator_transposed(self, eta_a, eta_b, lam, precision=WT_FP64, out=None):
        out = np.zeros(self.shape) if out is None else out
        _check(wt_apply_operator_transposed(self.handle, eta_a, eta_b, lam, out, precision))
        return out

    def adjoint_solve(self, eta_a, eta_b, rhs, lam=None, tol=0.0):
        lam = np.zeros(self.shape) if lam is None else lam
        st, info = wt_adjoint_solve(self.handle, eta_a, eta_b, rhs, lam, tol)
        _check(st)
        return lam, info

    def adjoint_step(self, dt, eta, u, w, lam_eta, lam_u, lam_w, dJ_dh=None):
        """Reverse one step from state (eta, u, w); lam_* and dJ_dh are updated in place."""
        _check(wt_adjoint_step(self.handle, dt, eta, u, w, lam_eta, lam_u, lam_w, dJ_dh))

    def autotune(self, eta_a, eta_b, rhs, reps=3):
        """Pick the fastest converging solver settings for this problem; returns
        (options dict, best ms, ms of the options on entry)."""
        st, o, best, entry = wt_autotune(self.handle, eta_a, eta_b, rhs, reps)
        _check(st)
        return {k: getattr(o, k) for k, _ in wt_options._fields_}, best, entry

    def step(self, dt, nsteps=1):
        _check(wt_step(self.handle, dt, nsteps))

    def stats(self):
        st, s, i = wt_get_stats(self.handle)
        _check(st)
        return s, i

    def profile(self, mask):
        _check(wt_profile(self.handle, mask))

    def profile_read(self, kernel_class):
        st, ms, n, b, f = wt_profile_read(self.handle, kernel_class)
        _check(st)
        return dict(ms=ms, launches=n, bytes=b, flops=f)

    def relax(self, x0, x1, eta_target=None, u_target=None, w_target=None, v_target=None):
        """Blend the state towards the targets inside the zone from x0 (weight 0)
        to x1 (weight 1)."""
        _check(wt_relax(self.handle, x0, x1, eta_target, u_target, v_target, w_target))

    def stream_function_wave(self, nwaves, H, nmodes=32, time=0.0):
        """(eta, u, w, c) of the stream-function wave at the tank's nodes (2D, flat bottom)."""
        eta = np.zeros((1, self.Nx))
        u, w = np.zeros(self.shape), np.zeros(self.shape)
        st, c = wt_stream_function_wave(self.handle, nwaves, H, nmodes, time, eta, u, w)
        _check(st)
        return eta, u, w, c

    def time_kernel(self, eta_a, eta_b, what=WT_TIME_OPERATOR, precision=WT_FP32, reps=200):
        """(ms per unit, kernels per unit) of the operator apply or the V-cycle,
        timed as one CUDA graph of `reps` units between two events."""
        st, ms, n = wt_time_kernel(self.handle, eta_a, eta_b, what, precision, reps)
        _check(st)
        return ms, n

    def launches(self):
        st, n = wt_get_launches(self.handle)
        _check(st)
        return n

    def close(self):
        if getattr(self, "handle", None) is not None:
            wt_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Owning wrapper of a wt_batch handle: independent 2D tanks of uneven
    size advanced together by one persistent kernel launch per ``step``."""

    def __init__(self, Nx, Nz, L, bathymetry, g=9.81, nu=0.0, **options):
        self.Nx = [int(v) for v in Nx]
        self.Nz = [int(v) for v in Nz]
        self.L = [float(v) for v in L]
        hs = [h if hasattr(h, "data_ptr") else np.ascontiguousarray(h, dtype=np.float64)
              for h in bathymetry]
        st, b = wt_create_batch(self.Nx, self.Nz, self.L, hs, g, nu)
        _check(st)
        self.handle = b
        if options:
            self.set_options(**options)

    def __len__(self):
        return len(self.Nx)

    def set_options(self, **kw):
        """Apply one option set to every tank of the batch: the keys given here
        on top of the library defaults (unlike Tank.set_options, which changes
        only the given keys of the tank's current options)."""
        o = wt_default_options()
        for k, v in kw.items():
            if k not in dict(wt_options._fields_):
                raise KeyError(k)
            setattr(o, k, v)
        _check(wt_batch_set_options(self.handle, o))

    def set_state(self, i, eta, u, w, time=0.0):
        _check(wt_batch_set_state(self.handle, i, eta, u, w, time))

    def get_state(self, i):
        M1, Nx = self.Nz[i] + 1, self.Nx[i]
        eta = np.zeros((1, Nx))
        u, w = np.zeros((M1, 1, Nx)), np.zeros((M1, 1, Nx))
        st, tm = wt_batch_get_state(self.handle, i, eta, u, w)
        _check(st)
        return eta, u, w, tm

    def step(self, dt, nsteps=1):
        dt = np.broadcast_to(np.asarray(dt, dtype=np.float64), (len(self),))
        _check(wt_batch_step(self.handle, dt, nsteps))

    def set_stream(self, stream_handle):
        _check(wt_batch_set_stream(self.handle, stream_handle))

    def options(self):
        st, o = wt_batch_get_options(self.handle)
        _check(st)
        return {k: getattr(o, k) for k, _ in wt_options._fields_}

    def autotune(self, dt, reps=1):
        """Pick omega and the sweep counts that minimise one batch step from the
        current states (restored); returns (options, best ms, entry ms)."""
        dt = np.broadcast_to(np.asarray(dt, dtype=np.float64), (len(self),))
        st, o, bm, em = wt_batch_autotune(self.handle, dt, reps)
        _check(st)
        return {k: getattr(o, k) for k, _ in wt_options._fields_}, bm, em

    def stats(self, i):
        st, s, it, r = wt_batch_stats(self.handle, i)
        _check(st)
        return s, it, r

    def close(self):
        if getattr(self, "handle", None) is not None:
            wt_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
