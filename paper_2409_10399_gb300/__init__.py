"""GB300 library of the six coupled Eulerian-Eulerian LBM schemes
(Piredda & Asinari, arXiv 2409.10399), Python binding.

The compute path is the CUDA library ``_build/liblbm.so`` behind the C ABI of
``include/lbm.h``; this module only marshals arguments (numpy host arrays or
torch CUDA tensors) into it.  There is no CPU fallback: if the library is not
built, or no GPU is present, the calls raise.
"""
import ctypes
import os
import threading

import numpy as np

from . import build as _build

__all__ = ["Simulation", "Batch", "Surrogate", "LBMError", "load_library", "lattice_tables", "tile_limit", "fno_gemm",
           "PRECISION", "LATTICE", "BC"]

LATTICE = {"D1Q3": 1, "D2Q9": 2, "D3Q19": 3}
PRECISION = {"fp64": 0, "fp32": 1, "fp16dev": 2, "fp64dev": 3, "fp16ab": 4}
BC = {"periodic": 0, "wall": 1, "inlet": 2, "outlet": 3}
ERRORS = {0: "LBM_OK", -1: "LBM_EINVAL", -2: "LBM_ENOMEM", -3: "LBM_ECUDA", -4: "LBM_ENAN",
          -5: "LBM_EDRIFT", -6: "LBM_ETIMEOUT", -7: "LBM_ESTATE"}


class LBMError(RuntimeError):
    def __init__(self, code, msg=""):
        self.code = code
        super().__init__("%s (%d)%s" % (ERRORS.get(code, "?"), code, (": " + msg) if msg else ""))


class Params(ctypes.Structure):
    """Mirror of ``lbm_params`` (include/lbm.h)."""
    _fields_ = [
        ("R", ctypes.c_double),
        ("omega_g", ctypes.c_double), ("omega_l", ctypes.c_double),
        ("omega_alpha", ctypes.c_double),
        ("psi_g", ctypes.c_double), ("psi_l", ctypes.c_double),
        ("drag_model", ctypes.c_int), ("kappa_I", ctypes.c_double), ("kappa_W", ctypes.c_double),
        ("g_hat", ctypes.c_double), ("g_axis", ctypes.c_int),
        ("gamma", ctypes.c_double), ("n_gamma", ctypes.c_int),
        ("spalding_mode", ctypes.c_int), ("alpha_floor", ctypes.c_double),
        ("bc_lo", ctypes.c_int * 3), ("bc_hi", ctypes.c_int * 3),
        ("inlet_lo", ctypes.c_int), ("inlet_hi", ctypes.c_int),
        ("in_alpha", ctypes.c_double * 2), ("in_ug", ctypes.c_double * 2), ("in_ul", ctypes.c_double * 2),
        ("ramp_nt", ctypes.c_int), ("inlet_ul_mode", ctypes.c_int),
        ("precision", ctypes.c_int), ("diag_every", ctypes.c_int), ("drift_limit", ctypes.c_double),
        ("beta_stencil", ctypes.c_int),
    ]


_LIB = None
_LOCK = threading.Lock()


def load_library(build_if_missing=True):
    """Load liblbm.so (building it with nvcc if it is missing or stale)."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        so = _build.SO
        if build_if_missing:
            so = _build.build()
        if not os.path.exists(so):
            raise RuntimeError("liblbm.so is not built; run paper_2409_10399_gb300.build.build()")
        lib = ctypes.CDLL(so)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        dp = ctypes.c_void_p  # double* (host or device address)
        sigs = {
            "lbm_default_params": (None, [ctypes.POINTER(Params)]),
            "lbm_lattice": (I, [I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(D)]),
            "lbm_create": (I, [I, I, I, I, I, ctypes.POINTER(Params), ctypes.POINTER(P)]),
            "lbm_init": (I, [P, dp, dp, dp, dp, I]),
            "lbm_step": (I, [P, I]),
            "lbm_get_moments": (I, [P, dp, dp, dp, dp, dp, dp, I]),
            "lbm_get_populations": (I, [P, I, dp, I]),
            "lbm_get_diag": (I, [P, ctypes.POINTER(D)]),
            "lbm_set_stream": (I, [P, P]),
            "lbm_time": (I, [P, ctypes.POINTER(ctypes.c_longlong)]),
            "lbm_set_graph": (I, [P, I]),
            "lbm_set_tile": (I, [P, I, I, I]),
            "lbm_get_tile": (I, [P, ctypes.POINTER(I)]),
            "lbm_tile_limit": (I, [I, I, ctypes.POINTER(I)]),
            "lbm_fno_create": (I, [I, I, I, I, I, ctypes.POINTER(P)]),
            "lbm_fno_num_params": (I, [P, ctypes.POINTER(ctypes.c_longlong)]),
            "lbm_fno_set_params": (I, [P, ctypes.POINTER(ctypes.c_float), ctypes.c_longlong]),
            "lbm_fno_get_params": (I, [P, ctypes.POINTER(ctypes.c_float), ctypes.c_longlong]),
            "lbm_fno_get_grads": (I, [P, ctypes.POINTER(ctypes.c_float), ctypes.c_longlong]),
            "lbm_fno_zero_grads": (I, [P]),
            "lbm_fno_set_norm": (I, [P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                     ctypes.POINTER(ctypes.c_float)]),
            "lbm_fno_set_stream": (I, [P, P]),
            "lbm_fno_accumulate": (I, [P, dp, dp, ctypes.POINTER(D)]),
            "lbm_fno_set_loss": (I, [P, D]),
            "lbm_fno_set_inflow": (I, [P, D]),
            "lbm_fno_adam": (I, [P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]),
            "lbm_fno_advance": (I, [P, dp, dp, D, ctypes.POINTER(D), ctypes.POINTER(I)]),
            "lbm_surrogate_advance": (I, [P, P, I, D, ctypes.POINTER(D), ctypes.POINTER(I)]),
            "lbm_fno_launch_count": (I, [P, ctypes.POINTER(ctypes.c_longlong)]),
            "lbm_fno_last_error": (ctypes.c_char_p, [P]),
            "lbm_fno_destroy": (I, [P]),
            "lbm_fno_gemm": (I, [I, I, I, I, I, ctypes.c_float, dp, I, ctypes.c_longlong, dp, I, ctypes.c_longlong,
                                 ctypes.c_float, dp, I, ctypes.c_longlong, I, I, I, P]),
            "lbm_launch_count": (I, [P, ctypes.POINTER(ctypes.c_longlong)]),
            "lbm_last_error": (ctypes.c_char_p, [P]),
            "lbm_destroy": (I, [P]),
            "lbm_diag_populations_noalloc": (I, [I, I, dp, ctypes.c_longlong, dp, I, P]),
            "lbm_batch_create": (I, [I, I, ctypes.POINTER(I), ctypes.POINTER(Params), ctypes.POINTER(P)]),
            "lbm_batch_size": (I, [P, ctypes.POINTER(I)]),
            "lbm_batch_init": (I, [P, I, dp, dp, dp, dp, I]),
            "lbm_batch_step": (I, [P, I]),
            "lbm_batch_get_moments": (I, [P, I, dp, dp, dp, dp, dp, dp, I]),
            "lbm_batch_get_diag": (I, [P, I, ctypes.POINTER(D)]),
            "lbm_batch_set_tile": (I, [P, I, I, I]),
            "lbm_batch_get_tile": (I, [P, ctypes.POINTER(I)]),
            "lbm_batch_set_graph": (I, [P, I]),
            "lbm_batch_set_stream": (I, [P, P]),
            "lbm_batch_time": (I, [P, ctypes.POINTER(ctypes.c_longlong)]),
            "lbm_batch_launch_count": (I, [P, ctypes.POINTER(ctypes.c_longlong)]),
            "lbm_batch_last_error": (ctypes.c_char_p, [P]),
            "lbm_batch_destroy": (I, [P]),
        }
        for name, (res, args) in sigs.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
        return lib


def lattice_tables(lattice):
    """(v[Q, D], w[Q]) of the library's velocity order (no GPU needed)."""
    lib = load_library()
    L = LATTICE[lattice]
    Q = ctypes.c_int()
    v = (ctypes.c_int * 57)()
    w = (ctypes.c_double * 19)()
    rc = lib.lbm_lattice(L, ctypes.byref(Q), v, w)
    if rc:
        raise LBMError(rc)
    q = Q.value
    return np.array(v[:3 * q], np.int64).reshape(q, 3)[:, :L], np.array(w[:q])


def tile_limit(lattice, precision):
    """Largest tile (threads per block) of the fused step kernel of `lattice`
    ("D2Q9" or its D) in `precision` ("fp32" ... or its code); no GPU needed."""
    L = LATTICE[lattice] if isinstance(lattice, str) else int(lattice)
    prec = PRECISION[precision] if isinstance(precision, str) else int(precision)
    m = ctypes.c_int()
    rc = load_library().lbm_tile_limit(L, prec, ctypes.byref(m))
    if rc:
        raise LBMError(rc, "lbm_tile_limit")
    return m.value


def default_params():
    p = Params()
    load_library().lbm_default_params(ctypes.byref(p))
    return p


def make_params(d):
    p = default_params()
    for k, v in d.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISION[v]
        if not hasattr(p, k):
            continue
        cur = getattr(p, k)
        if isinstance(cur, ctypes.Array):
            arr = type(cur)(*v)
            setattr(p, k, arr)
        elif isinstance(cur, int):
            setattr(p, k, int(v))
        else:
            setattr(p, k, float(v))
    return p


class Batch:
    """Many independent lattices of one type and precision advanced together
    (include/lbm.h, batched form).  ``Batch("D2Q9", [(nx, ny), ...],
    [params, ...])``; instance i is initialised with ``init(i, ...)``."""

    def __init__(self, lattice, dims_list, params_list):
        self._lib = load_library()
        self.lattice = lattice
        self.D = LATTICE[lattice]
        self.dims = [tuple(int(d) for d in dims) + (1,) * (3 - len(dims)) for dims in dims_list]
        n = len(self.dims)
        flat = (ctypes.c_int * (3 * n))(*[v for d in self.dims for v in d])
        self._params = (Params * n)(*[make_params(p) for p in params_list])
        h = ctypes.c_void_p()
        rc = self._lib.lbm_batch_create(self.D, n, flat, self._params, ctypes.byref(h))
        if rc:
            raise LBMError(rc, "lbm_batch_create")
        self._h = h
        self.n = n
        self._keep = {}

    def _check(self, rc, what):
        if rc:
            msg = self._lib.lbm_batch_last_error(self._h)
            raise LBMError(rc, "%s: %s" % (what, msg.decode() if msg else ""))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, i, alpha_g, u_g, u_l, p_k):
        N = int(np.prod(self.dims[i]))
        arrs = [np.ascontiguousarray(np.asarray(a, np.float64)) for a in (alpha_g, u_g, u_l, p_k)]
        for a, m in zip(arrs, (N, self.D * N, self.D * N, N)):
            if a.size != m:
                raise ValueError("field size %d, expected %d" % (a.size, m))
        self._check(self._lib.lbm_batch_init(self._h, int(i), *[ctypes.c_void_p(a.ctypes.data) for a in arrs], 0),
                    "lbm_batch_init")

    def step(self, n=1):
        self._check(self._lib.lbm_batch_step(self._h, int(n)), "lbm_batch_step")

    def set_tile(self, tx, ty=1, tz=1):
        self._check(self._lib.lbm_batch_set_tile(self._h, int(tx), int(ty), int(tz)), "lbm_batch_set_tile")

    @property
    def tile(self):
        t = (ctypes.c_int * 3)()
        self._check(self._lib.lbm_batch_get_tile(self._h, t), "lbm_batch_get_tile")
        return tuple(t)

    def set_graph(self, enable):
        self._check(self._lib.lbm_batch_set_graph(self._h, int(bool(enable))), "lbm_batch_set_graph")

    def set_stream(self, stream):
        handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream or 0)
        self._stream = stream
        self._check(self._lib.lbm_batch_set_stream(self._h, ctypes.c_void_p(handle)), "lbm_batch_set_stream")

    @property
    def t(self):
        v = ctypes.c_longlong()
        self._check(self._lib.lbm_batch_time(self._h, ctypes.byref(v)), "lbm_batch_time")
        return v.value

    @property
    def launches(self):
        v = ctypes.c_longlong()
        self._check(self._lib.lbm_batch_launch_count(self._h, ctypes.byref(v)), "lbm_batch_launch_count")
        return v.value

    def moments(self, i):
        N = int(np.prod(self.dims[i]))
        D = self.D
        res = dict(alpha_g=np.empty(N), u_g=np.empty((D, N)), u_l=np.empty((D, N)), p_k=np.empty(N),
                   S_g=np.empty(N), S_l=np.empty(N))
        ptrs = [ctypes.c_void_p(res[k].ctypes.data) for k in ("alpha_g", "u_g", "u_l", "p_k", "S_g", "S_l")]
        self._check(self._lib.lbm_batch_get_moments(self._h, int(i), *ptrs, 0), "lbm_batch_get_moments")
        return res

    def diag(self, i):
        out = (ctypes.c_double * 8)()
        self._check(self._lib.lbm_batch_get_diag(self._h, int(i), out), "lbm_batch_get_diag")
        return np.array(out[:])


def diag_populations_noalloc(lattice, spalding_mode, pops_ptr, n_nodes, out_ptr, out_on_device, stream=0):
    """Diagnostics of a caller-owned FP64 population buffer (device pointer
    `pops_ptr`, 6*Q*n_nodes doubles) into `out_ptr` (8 doubles) without any
    allocation; see lbm_diag_populations_noalloc in include/lbm.h."""
    lib = load_library()
    rc = lib.lbm_diag_populations_noalloc(LATTICE[lattice], int(spalding_mode), ctypes.c_void_p(pops_ptr),
                                          int(n_nodes), ctypes.c_void_p(out_ptr), int(out_on_device),
                                          ctypes.c_void_p(int(stream or 0)))
    if rc:
        raise LBMError(rc, "lbm_diag_populations_noalloc")


def _is_torch(x):
    return type(x).__module__.startswith("torch")


class Simulation:
    """One lattice run on the current CUDA device.

    ``Simulation("D2Q9", (nx, ny), params)`` where ``params`` is a dict of
    ``lbm_params`` fields (``precision`` may be "fp64", "fp32", "fp16dev").
    """

    def __init__(self, lattice, dims, params):
        self._lib = load_library()
        self.lattice = lattice
        self.D = LATTICE[lattice]
        dims = tuple(int(d) for d in dims) + (1,) * (3 - len(dims))
        self.dims = dims
        self.N = dims[0] * dims[1] * dims[2]
        self.params = make_params(params)
        h = ctypes.c_void_p()
        rc = self._lib.lbm_create(self.D, self.D, dims[0], dims[1], dims[2], ctypes.byref(self.params), ctypes.byref(h))
        if rc:
            raise LBMError(rc, "lbm_create(%s, %r)" % (lattice, dims))
        self._h = h
        self._stream = None

    def _check(self, rc, what):
        if rc:
            msg = self._lib.lbm_last_error(self._h)
            raise LBMError(rc, "%s: %s" % (what, msg.decode() if msg else ""))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_graph(self, enable):
        """Replay periods of steps from a CUDA graph (lbm_set_graph; default on)."""
        self._check(self._lib.lbm_set_graph(self._h, 1 if enable else 0), "lbm_set_graph")

    def set_stream(self, stream):
        """Use a torch.cuda.Stream (or a raw cudaStream_t int) for all work."""
        handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream or 0)
        self._stream = stream
        self._check(self._lib.lbm_set_stream(self._h, ctypes.c_void_p(handle)), "lbm_set_stream")

    def init(self, alpha_g, u_g, u_l, p_k):
        """Fields as numpy float64 (host) or torch float64 CUDA tensors."""
        arrs = [alpha_g, u_g, u_l, p_k]
        if all(_is_torch(a) and a.is_cuda for a in arrs):
            arrs = [a.contiguous() for a in arrs]
            for a in arrs:
                if a.dtype.__repr__() != "torch.float64":
                    raise TypeError("device fields must be float64")
            self._keep = arrs
            ptrs = [a.data_ptr() for a in arrs]
            on_dev = 1
        else:
            arrs = [np.ascontiguousarray(np.asarray(a, np.float64)) for a in arrs]
            sizes = [self.N, self.D * self.N, self.D * self.N, self.N]
            for a, n in zip(arrs, sizes):
                if a.size != n:
                    raise ValueError("field size %d, expected %d" % (a.size, n))
            self._keep = arrs
            ptrs = [a.ctypes.data for a in arrs]
            on_dev = 0
        self._check(self._lib.lbm_init(self._h, *[ctypes.c_void_p(p) for p in ptrs], on_dev), "lbm_init")

    def step(self, n=1):
        self._check(self._lib.lbm_step(self._h, int(n)), "lbm_step")

    def set_tile(self, tx, ty=1, tz=1):
        """Thread-block tile of the fused step (results do not depend on it)."""
        self._check(self._lib.lbm_set_tile(self._h, int(tx), int(ty), int(tz)), "lbm_set_tile")

    @property
    def tile(self):
        t = (ctypes.c_int * 3)()
        self._check(self._lib.lbm_get_tile(self._h, t), "lbm_get_tile")
        return tuple(t)

    @property
    def t(self):
        v = ctypes.c_longlong()
        self._check(self._lib.lbm_time(self._h, ctypes.byref(v)), "lbm_time")
        return v.value

    @property
    def launches(self):
        v = ctypes.c_longlong()
        self._check(self._lib.lbm_launch_count(self._h, ctypes.byref(v)), "lbm_launch_count")
        return v.value

    def moments(self, out=None, host_out=None):
        """dict of alpha_g, u_g (D, N), u_l (D, N), p_k, S_g, S_l.

        With ``out`` a dict of torch float64 CUDA tensors of those shapes, the
        library writes into them on the device; with ``host_out`` a dict of
        caller-owned (e.g. pinned) contiguous float64 numpy arrays it writes
        into those; otherwise it returns new numpy arrays."""
        N, D = self.N, self.D
        keys = ("alpha_g", "u_g", "u_l", "p_k", "S_g", "S_l")
        if host_out is not None:
            for k in keys:
                a = host_out.get(k)
                if a is not None and (a.dtype != np.float64 or not a.flags.c_contiguous):
                    raise TypeError("host_out[%s] must be contiguous float64" % k)
            ptrs = [ctypes.c_void_p(host_out[k].ctypes.data) if host_out.get(k) is not None else None for k in keys]
            self._check(self._lib.lbm_get_moments(self._h, *ptrs, 0), "lbm_get_moments")
            return host_out
        if out is not None:
            keys = ("alpha_g", "u_g", "u_l", "p_k", "S_g", "S_l")
            ptrs = [ctypes.c_void_p(out[k].data_ptr()) if k in out else None for k in keys]
            self._check(self._lib.lbm_get_moments(self._h, *ptrs, 1), "lbm_get_moments")
            return out
        res = dict(alpha_g=np.empty(N), u_g=np.empty((D, N)), u_l=np.empty((D, N)), p_k=np.empty(N),
                   S_g=np.empty(N), S_l=np.empty(N))
        ptrs = [ctypes.c_void_p(res[k].ctypes.data) for k in ("alpha_g", "u_g", "u_l", "p_k", "S_g", "S_l")]
        self._check(self._lib.lbm_get_moments(self._h, *ptrs, 0), "lbm_get_moments")
        return res

    def populations(self, s):
        """Full populations of scheme s as numpy (Q, N), library velocity order."""
        Q = {1: 3, 2: 9, 3: 19}[self.D]
        out = np.empty((Q, self.N))
        self._check(self._lib.lbm_get_populations(self._h, int(s), ctypes.c_void_p(out.ctypes.data), 0),
                    "lbm_get_populations")
        return out

    def diag(self):
        out = (ctypes.c_double * 8)()
        self._check(self._lib.lbm_get_diag(self._h, out), "lbm_get_diag")
        return np.array(out[:])


def _f32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


class Surrogate:
    """The learned 2D surrogate (include/lbm.h, lbm_fno_*): a factorised
    Fourier neural operator over an nx x ny D2Q9 state.  States are torch
    float64 CUDA tensors of shape (6, nx*ny): alpha_g, u_g (x, y), u_l (x, y),
    p_k."""

    def __init__(self, nx, ny, channels=64, modes=32, layers=4):
        self._lib = load_library()
        h = ctypes.c_void_p()
        rc = self._lib.lbm_fno_create(int(nx), int(ny), int(channels), int(modes), int(layers), ctypes.byref(h))
        if rc:
            raise LBMError(rc, "lbm_fno_create(%d, %d, %d, %d, %d)" % (nx, ny, channels, modes, layers))
        self._h = h
        self.nx, self.ny, self.channels, self.modes, self.layers = nx, ny, channels, modes, layers
        n = ctypes.c_longlong()
        self._lib.lbm_fno_num_params(h, ctypes.byref(n))
        self.num_params = n.value

    def _check(self, rc, what):
        if rc:
            msg = self._lib.lbm_fno_last_error(self._h)
            raise LBMError(rc, "%s: %s" % (what, msg.decode() if msg else ""))

    def set_stream(self, stream):
        self._check(self._lib.lbm_fno_set_stream(self._h, ctypes.c_void_p(stream.cuda_stream)), "lbm_fno_set_stream")

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        if p.size != self.num_params:
            raise ValueError("expected %d parameters" % self.num_params)
        self._check(self._lib.lbm_fno_set_params(self._h, _f32p(p), p.size), "lbm_fno_set_params")

    def params(self):
        p = np.empty(self.num_params, np.float32)
        self._check(self._lib.lbm_fno_get_params(self._h, _f32p(p), p.size), "lbm_fno_get_params")
        return p

    def grads(self):
        g = np.empty(self.num_params, np.float32)
        self._check(self._lib.lbm_fno_get_grads(self._h, _f32p(g), g.size), "lbm_fno_get_grads")
        return g

    def zero_grads(self):
        self._check(self._lib.lbm_fno_zero_grads(self._h), "lbm_fno_zero_grads")

    def set_norm(self, mean, std_in, std_out):
        a = [np.ascontiguousarray(v, dtype=np.float32) for v in (mean, std_in, std_out)]
        self._norm = a
        self._check(self._lib.lbm_fno_set_norm(self._h, *[_f32p(v) for v in a]), "lbm_fno_set_norm")

    @staticmethod
    def _state(t):
        if not (_is_torch(t) and t.is_cuda and t.dtype.is_floating_point and t.element_size() == 8 and t.is_contiguous()):
            raise ValueError("states are contiguous float64 CUDA tensors of shape (6, nx*ny)")
        return ctypes.c_void_p(t.data_ptr())

    def set_loss(self, cons_weight):
        """Weight of the conservation term of the loss (lbm_fno_set_loss)."""
        self._check(self._lib.lbm_fno_set_loss(self._h, float(cons_weight)), "lbm_fno_set_loss")

    def set_inflow(self, dV):
        """Expected change of sum(alpha_g) over one call, the inlet's gas
        (lbm_fno_set_inflow); the volume check tests the change beyond it."""
        self._check(self._lib.lbm_fno_set_inflow(self._h, float(dV)), "lbm_fno_set_inflow")

    def accumulate(self, now, nxt):
        loss = ctypes.c_double()
        self._check(self._lib.lbm_fno_accumulate(self._h, self._state(now), self._state(nxt), ctypes.byref(loss)),
                    "lbm_fno_accumulate")
        return loss.value

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, grad_scale=1.0):
        self._check(self._lib.lbm_fno_adam(self._h, float(lr), float(beta1), float(beta2), float(eps),
                                           float(grad_scale)), "lbm_fno_adam")

    def advance(self, now, out, max_drift=1e-4):
        """out = surrogate(now); returns (drift, ok)."""
        d = ctypes.c_double()
        ok = ctypes.c_int()
        self._check(self._lib.lbm_fno_advance(self._h, self._state(now), self._state(out), float(max_drift),
                                              ctypes.byref(d), ctypes.byref(ok)), "lbm_fno_advance")
        return d.value, bool(ok.value)

    def advance_lattice(self, sim, window=64, max_drift=1e-4):
        """One window on a live Simulation (lbm_surrogate_advance): the
        surrogate's state when its check passes, else `window` LBM steps;
        returns (drift, used)."""
        d = ctypes.c_double()
        used = ctypes.c_int()
        rc = self._lib.lbm_surrogate_advance(sim._h, self._h, int(window), float(max_drift), ctypes.byref(d),
                                             ctypes.byref(used))
        if rc != 0:
            msgs = [self._lib.lbm_last_error(sim._h), self._lib.lbm_fno_last_error(self._h)]
            raise LBMError(rc, "lbm_surrogate_advance: " + "; ".join(m.decode() for m in msgs if m))
        return d.value, bool(used.value)

    @property
    def launches(self):
        n = ctypes.c_longlong()
        self._lib.lbm_fno_launch_count(self._h, ctypes.byref(n))
        return n.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_fno_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fno_gemm(A, B, C, ta=False, tb=False, alpha=1.0, beta=0.0, batch=1, sA=0, sB=0, sC=0, ksplit=1, M=None,
             N=None, K=None, lda=None, ldb=None, ldc=None, stream=None):
    """The surrogate's BF16 matrix product (lbm_fno_gemm) on torch CUDA
    tensors: A, B bfloat16, C float32 or bfloat16 (2D row-major, or 3D with
    the batch first)."""
    lib = load_library()
    a2, b2, c2 = (t if t.dim() == 2 else t[0] for t in (A, B, C))
    M = M if M is not None else c2.shape[0]
    N = N if N is not None else c2.shape[1]
    K = K if K is not None else (a2.shape[0] if ta else a2.shape[1])
    lda = lda if lda is not None else a2.stride(0)
    ldb = ldb if ldb is not None else b2.stride(0)
    ldc = ldc if ldc is not None else c2.stride(0)
    if batch > 1:
        sA = sA or (A.stride(0) if A.dim() == 3 else 0)
        sB = sB or (B.stride(0) if B.dim() == 3 else 0)
        sC = sC or (C.stride(0) if C.dim() == 3 else 0)
    import torch
    out_f32 = 1 if C.dtype == torch.float32 else 0
    st = ctypes.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
    rc = lib.lbm_fno_gemm(int(ta), int(tb), M, N, K, float(alpha), ctypes.c_void_p(A.data_ptr()), lda, sA,
                          ctypes.c_void_p(B.data_ptr()), ldb, sB, float(beta), ctypes.c_void_p(C.data_ptr()), ldc, sC,
                          batch, out_f32, int(ksplit), st)
    if rc:
        raise LBMError(rc, "lbm_fno_gemm")
