"""ctypes binding of the C ABI in include/pint.h (argument marshalling only).

Every computation runs in libpint.so's CUDA kernels; this module only turns
Python arguments into the C structs and pointers the ABI takes.  Device
buffers are torch CUDA tensors (float64, or complex128 for frequency
vectors), passed by their data pointers; host buffers are numpy arrays.
Importing this module does not load the library; the first call does, and it
raises if libpint.so has not been built.
"""
import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpint.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "pint.h")

PINT_STOKES, PINT_OSEEN = 0, 1
PINT_WIND_NONE, PINT_WIND_RECIRC = 0, 1
PINT_PREC_FP64, PINT_PREC_FP32 = 0, 1
STATUS = {0: "PINT_OK", 1: "PINT_ERR_ARG", 2: "PINT_ERR_OOM", 3: "PINT_ERR_CUDA", 4: "PINT_ERR_NOT_CONVERGED",
          5: "PINT_ERR_NONFINITE", 6: "PINT_ERR_TIMEOUT", 7: "PINT_ERR_STATE"}
COMPONENT = {"mg_W": 0, "mg_Q": 1, "mg_QH": 2, "mg_Kp": 3, "cheb_M": 4, "cheb_Mp": 5, "block_prec": 6}


class Params(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("level", ctypes.c_int), ("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("n_t", ctypes.c_int), ("tau", ctypes.c_double), ("beta", ctypes.c_double), ("nu", ctypes.c_double),
                ("wind", ctypes.c_int), ("prec", ctypes.c_int), ("outer_restart", ctypes.c_int),
                ("outer_maxit", ctypes.c_int), ("outer_tol", ctypes.c_double), ("inner_tol", ctypes.c_double),
                ("inner_maxit", ctypes.c_int), ("mg_cycles", ctypes.c_int), ("mg_pre", ctypes.c_int),
                ("mg_post", ctypes.c_int), ("cheb_steps", ctypes.c_int), ("uzawa_steps", ctypes.c_int),
                ("uzawa_mu", ctypes.c_double), ("sor_omega", ctypes.c_double), ("fixed_inner_its", ctypes.c_int),
                ("linear", ctypes.c_int), ("dft_mode", ctypes.c_int), ("sor_omega_conv", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("outer_iterations", ctypes.c_int), ("restarts", ctypes.c_int), ("relres", ctypes.c_double),
                ("relres_history", ctypes.c_double * 256), ("inner_iterations_total", ctypes.c_int),
                ("inner_iterations_max", ctypes.c_int), ("precond_applies", ctypes.c_int),
                ("ms_precond", ctypes.c_double), ("ms_matvec", ctypes.c_double), ("ms_orth", ctypes.c_double),
                ("ms_total", ctypes.c_double)]


class Sizes(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("n_t", ctypes.c_int), ("J", ctypes.c_int), ("n_s", ctypes.c_size_t),
                ("n_q", ctypes.c_size_t), ("n_blk", ctypes.c_size_t), ("kkt_len", ctypes.c_size_t),
                ("freq_len", ctypes.c_size_t), ("device_bytes", ctypes.c_size_t)]


PROF_CLASSES = ["mg_q2", "mg_q1", "cheb", "dft_fwd", "dft_inv", "block_mv", "combo", "inner", "kkt_mv", "outer",
                "other", "apply"]
# kernel classes whose launches make up a preconditioner apply
APPLY_CLASSES = ["mg_q2", "mg_q1", "cheb", "dft_fwd", "dft_inv", "block_mv", "combo", "inner"]


class Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong * 12), ("timed", ctypes.c_longlong * 12),
                ("ms", ctypes.c_double * 12), ("bytes", ctypes.c_double * 12), ("host_syncs", ctypes.c_longlong)]


def _profile_dict(p):
    """Per-class counters, plus the host synchronisations under "host_syncs"."""
    out = {c: {"launches": p.launches[i], "timed": p.timed[i], "ms": p.ms[i], "bytes": p.bytes[i]}
           for i, c in enumerate(PROF_CLASSES)}
    out["host_syncs"] = p.host_syncs
    return out


_lib = None
_P = ctypes.c_void_p
class ServerParams(ctypes.Structure):
    _fields_ = [("device_budget", ctypes.c_size_t), ("max_active", ctypes.c_int), ("share_solves", ctypes.c_int)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong), ("failed", ctypes.c_longlong),
                ("active", ctypes.c_longlong), ("queued", ctypes.c_longlong), ("budget_bytes", ctypes.c_size_t),
                ("bytes_in_use", ctypes.c_size_t), ("bytes_peak", ctypes.c_size_t), ("active_peak", ctypes.c_int),
                ("shared_batches", ctypes.c_longlong), ("shared_member_solves", ctypes.c_longlong),
                ("shared_frequencies", ctypes.c_longlong), ("shared_max_members", ctypes.c_int)]


_SIGS = {
    "pint_default_params": (None, [ctypes.POINTER(Params)]),
    "pint_create": (ctypes.c_int, [ctypes.POINTER(Params), _P, ctypes.POINTER(_P)]),
    "pint_destroy": (ctypes.c_int, [_P]),
    "pint_get_sizes": (ctypes.c_int, [_P, ctypes.POINTER(Sizes)]),
    "pint_create_wind": (ctypes.c_int, [ctypes.POINTER(Params), _P, _P, ctypes.POINTER(_P)]),
    "pint_set_data": (ctypes.c_int, [_P, _P, _P, _P]),
    "pint_set_data_dirichlet": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "pint_get_rhs": (ctypes.c_int, [_P, _P]),
    "pint_kkt_matvec": (ctypes.c_int, [_P, _P, _P]),
    "pint_apply_preconditioner": (ctypes.c_int, [_P, _P, _P]),
    "pint_solve": (ctypes.c_int, [_P, _P, ctypes.POINTER(SolveInfo)]),
    "pint_solve_host": (ctypes.c_int, [_P, _P, ctypes.POINTER(SolveInfo)]),
    "pint_dft_forward": (ctypes.c_int, [_P, _P, _P]),
    "pint_dft_inverse": (ctypes.c_int, [_P, _P, _P]),
    "pint_freq_block_matvec": (ctypes.c_int, [_P, _P, _P]),
    "pint_freq_block_solve": (ctypes.c_int, [_P, _P, _P, _P]),
    "pint_component_apply": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P]),
    "pint_mg_apply_noalloc": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P]),
    "pint_mg_launch_config": (ctypes.c_int, [ctypes.c_int, ctypes.c_int]),
    "pint_profile_enable": (ctypes.c_int, [_P, ctypes.c_uint]),
    "pint_profile_read": (ctypes.c_int, [_P, ctypes.POINTER(Profile)]),
    "pint_debug_inject": (ctypes.c_int, [_P, ctypes.c_int]),
    "pint_convection_stencils": (ctypes.c_int, [ctypes.POINTER(Params), _P, ctypes.c_int, _P, _P]),
    "pint_estimate_device_bytes": (ctypes.c_size_t, [ctypes.POINTER(Params)]),
    "pint_autotune": (None, [ctypes.c_int]),
    "pint_autotune_report": (ctypes.c_size_t, [ctypes.c_char_p, ctypes.c_size_t]),
    "pint_server_create": (ctypes.c_int, [ctypes.POINTER(ServerParams), ctypes.POINTER(_P)]),
    "pint_group_create": (ctypes.c_int, [ctypes.POINTER(_P)]),
    "pint_create_in_group": (ctypes.c_int, [_P, ctypes.POINTER(Params), _P, ctypes.POINTER(_P)]),
    "pint_group_get_stats": (ctypes.c_int, [_P, _P]),
    "pint_group_destroy": (ctypes.c_int, [_P]),
    "pint_group_profile_enable": (ctypes.c_int, [_P, ctypes.c_uint]),
    "pint_group_profile_read": (ctypes.c_int, [_P, _P]),
    "pint_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(Params), _P, _P, _P, ctypes.POINTER(ctypes.c_longlong)]),
    "pint_server_wait": (ctypes.c_int, [_P, ctypes.c_longlong, _P, ctypes.POINTER(SolveInfo),
                                        ctypes.POINTER(ctypes.c_double)]),
    "pint_server_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(ServerStats)]),
    "pint_server_destroy": (ctypes.c_int, [_P]),
    "pint_server_last_error": (ctypes.c_char_p, []),
    "pint_last_error": (ctypes.c_char_p, [_P]),
}


def header_functions():
    """Names of the functions include/pint.h declares."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pint_[a-z0-9_]+)\s*\(", txt)))


def lib():
    """Load libpint.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libpint.so not found: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class PintError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def _check(code, handle=None):
    if code != 0:
        msg = lib().pint_last_error(handle)
        raise PintError(code, msg.decode() if msg else "")
    return code


def _dptr(t, dtype_name, numel=None):
    """Device pointer of a contiguous CUDA tensor of the given dtype."""
    if not hasattr(t, "data_ptr") or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if str(t.dtype) != "torch." + dtype_name:
        raise TypeError(f"expected torch.{dtype_name}, got {t.dtype}")
    if not t.is_contiguous():
        raise TypeError("expected a contiguous tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"expected {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a, numel=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if numel is not None and a.size != numel:
        raise ValueError(f"expected {numel} values, got {a.size}")
    return a


def default_params(**kw):
    p = Params()
    lib().pint_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


class Problem:
    """One discrete control problem on the GPU (handle of the C ABI)."""

    def __init__(self, params, stream=None, wind=None, group=None):
        """wind: for params.wind = PINT_WIND_NODAL (3), the wind's values at
        the finest Q2 nodes, shape (2, (2N+1)^2).  group: a Group whose
        handles share their frequency solves (pint_create_in_group)."""
        self.params = params
        h = ctypes.c_void_p()
        st = ctypes.c_void_p(stream) if stream else None
        if group is not None:
            _check(lib().pint_create_in_group(group.h, ctypes.byref(params), st, ctypes.byref(h)))
        elif wind is None:
            _check(lib().pint_create(ctypes.byref(params), st, ctypes.byref(h)))
        else:
            n2 = 2 * 2 ** params.level + 1
            w = _hptr(wind, 2 * n2 * n2)
            _check(lib().pint_create_wind(ctypes.byref(params), w.ctypes.data_as(ctypes.c_void_p), st,
                                          ctypes.byref(h)))
        self.h = h
        s = Sizes()
        _check(lib().pint_get_sizes(self.h, ctypes.byref(s)), self.h)
        self.sizes = s

    def close(self):
        if self.h:
            lib().pint_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # shapes
    @property
    def kkt_len(self):
        return self.sizes.kkt_len

    @property
    def freq_len(self):
        return self.sizes.freq_len

    def set_data(self, vd, f=None, v0=None):
        K, ns = self.sizes.n_t, self.sizes.n_s
        vd = _hptr(vd, K * 2 * ns)
        f = _hptr(f, K * 2 * ns)
        v0 = _hptr(v0, 2 * ns)
        ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p) if a is not None else None
        _check(lib().pint_set_data(self.h, ptr(vd), ptr(f), ptr(v0)), self.h)

    def set_data_dirichlet(self, vd, f=None, v0=None, g=None):
        """Data with a prescribed boundary velocity g (Sec. 5 problems); full-grid loads."""
        K, ns = self.sizes.n_t, self.sizes.n_s
        vd = _hptr(vd, K * 2 * ns)
        f = _hptr(f, K * 2 * ns)
        v0 = _hptr(v0, 2 * ns)
        g = _hptr(g, K * 2 * ns)
        ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p) if a is not None else None
        _check(lib().pint_set_data_dirichlet(self.h, ptr(vd), ptr(f), ptr(v0), ptr(g)), self.h)

    def get_rhs(self, b):
        _check(lib().pint_get_rhs(self.h, _dptr(b, "float64", self.kkt_len)), self.h)

    def kkt_matvec(self, x, y):
        _check(lib().pint_kkt_matvec(self.h, _dptr(x, "float64", self.kkt_len), _dptr(y, "float64", self.kkt_len)),
               self.h)

    def apply_preconditioner(self, r, z):
        _check(lib().pint_apply_preconditioner(self.h, _dptr(r, "float64", self.kkt_len),
                                               _dptr(z, "float64", self.kkt_len)), self.h)

    def solve(self, x, check=True):
        info = SolveInfo()
        code = lib().pint_solve(self.h, _dptr(x, "float64", self.kkt_len), ctypes.byref(info))
        if check:
            _check(code, self.h)
        return info

    def solve_host(self, x, check=True):
        a = np.ascontiguousarray(x, dtype=np.float64)
        if a.size != self.kkt_len or a is not x:
            raise ValueError("x must be a contiguous float64 array of kkt_len values")
        info = SolveInfo()
        code = lib().pint_solve_host(self.h, a.ctypes.data_as(ctypes.c_void_p), ctypes.byref(info))
        if check:
            _check(code, self.h)
        return info

    def dft_forward(self, x, xhat):
        _check(lib().pint_dft_forward(self.h, _dptr(x, "float64", self.kkt_len),
                                      _dptr(xhat, "complex128", self.freq_len)), self.h)

    def dft_inverse(self, xhat, x):
        _check(lib().pint_dft_inverse(self.h, _dptr(xhat, "complex128", self.freq_len),
                                      _dptr(x, "float64", self.kkt_len)), self.h)

    def freq_block_matvec(self, xhat, yhat):
        _check(lib().pint_freq_block_matvec(self.h, _dptr(xhat, "complex128", self.freq_len),
                                            _dptr(yhat, "complex128", self.freq_len)), self.h)

    def freq_block_solve(self, rhat, yhat):
        its = (ctypes.c_int * self.sizes.J)()
        _check(lib().pint_freq_block_solve(self.h, _dptr(rhat, "complex128", self.freq_len),
                                           _dptr(yhat, "complex128", self.freq_len), its), self.h)
        return list(its)

    def debug_inject(self, what=1):
        """Failure injection for tests (1: the next tensor-core DFT's bounded wait runs out)."""
        _check(lib().pint_debug_inject(self.h, int(what)), self.h)

    def mg_apply_noalloc(self, which, j, x, y):
        """Multigrid on one field with the library's fixed scratch array (no
        allocation).  Asynchronous on the handle's stream: x and y must stay
        valid, and y unread, until that stream is synchronised."""
        w = COMPONENT[which] if isinstance(which, str) else int(which)
        n = component_len(self.sizes, w)
        _check(lib().pint_mg_apply_noalloc(self.h, w, j, _dptr(x, "complex128", n), _dptr(y, "complex128", n)),
               self.h)

    def profile_enable(self, classes=()):
        """Reset the counters; time the named kernel classes with CUDA events."""
        mask = 0
        for c in classes:
            mask |= 1 << PROF_CLASSES.index(c)
        _check(lib().pint_profile_enable(self.h, mask), self.h)

    def profile_read(self):
        p = Profile()
        _check(lib().pint_profile_read(self.h, ctypes.byref(p)), self.h)
        return _profile_dict(p)

    def component_apply(self, which, j, x, y):
        w = COMPONENT[which] if isinstance(which, str) else int(which)
        n = component_len(self.sizes, w)
        _check(lib().pint_component_apply(self.h, w, j, _dptr(x, "complex128", n), _dptr(y, "complex128", n)),
               self.h)


def component_len(sizes, which):
    """Complex values of one component's input and output field: n_q for the
    pressure operators (3, 5), n_blk for a whole frequency block (6), else n_s."""
    if which in (3, 5):
        return int(sizes.n_q)
    if which == 6:
        return int(sizes.n_blk)
    return int(sizes.n_s)


def convection_stencils(params, level_index=0, wind=None):
    """(q2, q1): the FP64 node-order convection stencils the library builds
    for the two-vortex or nodal wind on one multigrid level (host only)."""
    n = 2 ** (params.level - level_index)
    q2 = np.zeros(((2 * n + 1) ** 2, 25))
    q1 = np.zeros(((n + 1) ** 2, 9))
    n2 = 2 * 2 ** params.level + 1
    w = _hptr(wind, 2 * n2 * n2)
    wp = w.ctypes.data_as(ctypes.c_void_p) if w is not None else None
    _check(lib().pint_convection_stencils(ctypes.byref(params), wp, level_index,
                                          q2.ctypes.data_as(ctypes.c_void_p), q1.ctypes.data_as(ctypes.c_void_p)))
    return q2, q1


def autotune(on=True):
    """Switch the multigrid CTA-size autotuner on or off (process-wide)."""
    lib().pint_autotune(1 if on else 0)


def mg_launch_config(threads=0, staging=-1):
    """Multigrid launch choice while the tuner is off (see pint.h)."""
    _check(lib().pint_mg_launch_config(int(threads), int(staging)), None)


def autotune_report():
    """The autotuner's decisions, one launch shape per line."""
    n = lib().pint_autotune_report(None, 0)
    buf = ctypes.create_string_buffer(n)
    lib().pint_autotune_report(buf, n)
    return buf.value.decode()


def estimate_device_bytes(params):
    """Upper estimate of the device memory a handle for these parameters holds."""
    return int(lib().pint_estimate_device_bytes(ctypes.byref(params)))


class GroupStats(ctypes.Structure):
    _fields_ = [("batches", ctypes.c_longlong), ("member_solves", ctypes.c_longlong),
                ("frequencies", ctypes.c_longlong), ("max_members", ctypes.c_int)]


class Group:
    """Handles whose frequency solves run in shared launches when they solve
    concurrently (pint_group_*); close it after its handles."""

    def __init__(self):
        h = ctypes.c_void_p()
        _check(lib().pint_group_create(ctypes.byref(h)))
        self.h = h

    def profile_enable(self, classes=()):
        """Reset the shared solves' counters; time the named kernel classes."""
        mask = 0
        for c in classes:
            mask |= 1 << PROF_CLASSES.index(c)
        _check(lib().pint_group_profile_enable(self.h, mask))

    def profile_read(self):
        p = Profile()
        _check(lib().pint_group_profile_read(self.h, ctypes.byref(p)))
        return _profile_dict(p)

    def stats(self):
        st = GroupStats()
        _check(lib().pint_group_get_stats(self.h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in GroupStats._fields_}

    def close(self):
        if self.h:
            lib().pint_group_destroy(self.h)
            self.h = None


class Server:
    """Serving loop (pint_server_*): continuous batching of control problems
    on the current device; see include/pint.h."""

    def __init__(self, max_active=4, device_budget=0, share_solves=False):
        sp = ServerParams(device_budget, max_active, 1 if share_solves else 0)
        h = ctypes.c_void_p()
        code = lib().pint_server_create(ctypes.byref(sp), ctypes.byref(h))
        if code != 0:
            raise PintError(code, lib().pint_server_last_error().decode())
        self.h = h

    def submit(self, params, vd, f=None, v0=None):
        """Queue a request (host arrays are copied); returns its id."""
        n_s = (2 * (1 << params.level) + 1) ** 2
        keep = [np.ascontiguousarray(vd, dtype=np.float64).reshape(params.n_t * 2 * n_s)]
        ptrs = [keep[0].ctypes.data_as(ctypes.c_void_p)]
        for a, n in ((f, params.n_t * 2 * n_s), (v0, 2 * n_s)):
            if a is None:
                ptrs.append(None)
            else:
                keep.append(np.ascontiguousarray(a, dtype=np.float64).reshape(n))
                ptrs.append(keep[-1].ctypes.data_as(ctypes.c_void_p))
        rid = ctypes.c_longlong()
        code = lib().pint_server_submit(self.h, ctypes.byref(params), ptrs[0], ptrs[1], ptrs[2], ctypes.byref(rid))
        if code != 0:
            raise PintError(code, lib().pint_server_last_error().decode())
        return rid.value

    def wait(self, rid, kkt_len, check=True):
        """Block until request rid completes: (x, info, latency_ms, status)."""
        x = np.zeros(kkt_len)
        info = SolveInfo()
        lat = ctypes.c_double()
        code = lib().pint_server_wait(self.h, rid, x.ctypes.data_as(ctypes.c_void_p), ctypes.byref(info),
                                      ctypes.byref(lat))
        if check and code != 0:
            raise PintError(code, lib().pint_server_last_error().decode())
        return x, info, lat.value, code

    def stats(self):
        st = ServerStats()
        lib().pint_server_get_stats(self.h, ctypes.byref(st))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if self.h:
            lib().pint_server_destroy(self.h)
            self.h = None

    def __del__(self):
        # finish the workers before the interpreter tears down the CUDA context
        try:
            self.close()
        except Exception:
            pass
