"""FP64 CPU oracle of the six coupled EE-LBM schemes (arXiv 2409.10399, Sec. 2-3).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library under ``paper_2409_10399_gb300/`` and imports nothing
from it; the only module both sides use is the seeded input generator
``lbm_inputs``.

``Oracle`` wraps ``lbm_oracle.c`` (plain C, FP64, two-array push streaming).
``brute`` is an independent pure-Python stepper for tiny lattices, ``fd`` the
finite-difference solver of Sec. 3.4, ``params`` the similarity helper of
Sec. 3.3.  Parity status of each part is listed in ``PARITY`` below.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liblbm_oracle.so")
_LOCK = threading.Lock()

# Which functions are pinned by what (see tests/test_oracle_*.py).
PARITY = {
    "equilibria": "pinned: App. A D1Q3 formulas, moment identities (Sec. 2.1.1, 2.2)",
    "collision+stream": "pinned: uniform fixed point, homogeneous ODE limit and steady state, "
                        "conservation, mirror symmetry, D2Q9/D3Q19 -> D1Q3 projection, brute force",
    "inlet/outlet": "pinned: TEST #1 outlet values (Sec. 3.6)",
    "stabilisers": "pinned: Ohwada dashpot (sign, third liquid strategy) and the n_gamma latch phase against "
                   "the homogeneous-state recurrence of Eqs. (lbm-cont-g1Dhat), (lbm-cont-l1Dhat), "
                   "(lbm-cont-1D-update) (Sec. 3.2)",
    "fd": "partial: agreement with the LBM is qualitative in the paper (Sec. 3.6)",
}


def build(force=False):
    """Compile lbm_oracle.c into a shared library (gcc, FP64, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    src = os.path.join(_HERE, "lbm_oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-std=c11", "-o", tmp, src, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


class _Params(ctypes.Structure):
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
    ]


_lib = None


def _load():
    global _lib
    with _LOCK:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            dp = ctypes.POINTER(ctypes.c_double)
            lib.orc_create.restype = P
            lib.orc_create.argtypes = [ctypes.c_int] * 4 + [ctypes.POINTER(_Params)]
            lib.orc_destroy.argtypes = [P]
            lib.orc_set_threads.argtypes = [P, ctypes.c_int]
            lib.orc_Q.argtypes = [P]
            lib.orc_Q.restype = ctypes.c_int
            lib.orc_time.argtypes = [P]
            lib.orc_time.restype = ctypes.c_long
            lib.orc_lattice.argtypes = [P, ctypes.POINTER(ctypes.c_int), dp, ctypes.POINTER(ctypes.c_int)]
            lib.orc_init.argtypes = [P, dp, dp, dp, dp]
            lib.orc_step.argtypes = [P, ctypes.c_long]
            lib.orc_moments.argtypes = [P, dp, dp, dp, dp, dp, dp]
            lib.orc_get_pops.argtypes = [P, ctypes.c_int, dp]
            lib.orc_set_pops.argtypes = [P, ctypes.c_int, dp]
            lib.orc_get_held.argtypes = [P, dp, dp, dp]
            lib.orc_diag.argtypes = [P, dp]
            lib.orc_equilibria.argtypes = [P, ctypes.c_double, ctypes.c_double, dp, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_double, dp, dp, dp, dp]
            _lib = lib
    return _lib


PARAM_DEFAULTS = dict(
    R=2.0, omega_g=1.0, omega_l=1.0, omega_alpha=1.5, psi_g=0.0, psi_l=0.0,
    drag_model=0, kappa_I=0.0, kappa_W=0.0, g_hat=0.0, g_axis=0, gamma=0.0, n_gamma=1,
    spalding_mode=2, alpha_floor=1e-8, bc_lo=(0, 0, 0), bc_hi=(0, 0, 0), inlet_lo=0, inlet_hi=0,
    in_alpha=(0.0, 0.0), in_ug=(0.0, 0.0), in_ul=(0.0, 0.0), ramp_nt=0, inlet_ul_mode=0,
)


def _mk_params(d):
    p = dict(PARAM_DEFAULTS)
    for k, v in d.items():
        if k in p:
            p[k] = v
    s = _Params()
    for k, v in p.items():
        if k in ("bc_lo", "bc_hi"):
            arr = (ctypes.c_int * 3)(*[int(x) for x in v])
            setattr(s, k, arr)
        elif k in ("in_alpha", "in_ug", "in_ul"):
            setattr(s, k, (ctypes.c_double * 2)(*[float(x) for x in v]))
        elif k in ("drag_model", "g_axis", "n_gamma", "spalding_mode", "inlet_lo", "inlet_hi",
                   "ramp_nt", "inlet_ul_mode"):
            setattr(s, k, int(v))
        else:
            setattr(s, k, float(v))
    return s


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


LATTICE_D = {"D1Q3": 1, "D2Q9": 2, "D3Q19": 3}


class Oracle:
    """One oracle run: ``Oracle(lattice, (nx, ny, nz), params)``.

    Fields are float64 arrays with node index x + nx*(y + ny*z); vector fields
    have shape (D, N).
    """

    def __init__(self, lattice, dims, params, threads=1):
        lib = _load()
        self.lattice = lattice
        self.D = LATTICE_D[lattice]
        dims = tuple(int(d) for d in dims) + (1,) * (3 - len(dims))
        self.dims = dims
        self.N = dims[0] * dims[1] * dims[2]
        self._p = _mk_params(params)
        self._h = lib.orc_create(self.D, dims[0], dims[1], dims[2], ctypes.byref(self._p))
        if not self._h:
            raise ValueError("oracle: invalid lattice or sizes %r %r" % (lattice, dims))
        self.Q = lib.orc_Q(self._h)
        lib.orc_set_threads(self._h, int(threads))

    def close(self):
        if self._h:
            _load().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_threads(self, n):
        _load().orc_set_threads(self._h, int(n))

    @property
    def t(self):
        return _load().orc_time(self._h)

    def lattice_tables(self):
        v = np.zeros(3 * self.Q, np.int32)
        w = np.zeros(self.Q)
        opp = np.zeros(self.Q, np.int32)
        _load().orc_lattice(self._h, v.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dptr(w),
                            opp.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        return v.reshape(self.Q, 3)[:, :self.D].copy(), w, opp

    def init(self, alpha_g, u_g, u_l, p_k):
        N, D = self.N, self.D
        a = np.ascontiguousarray(alpha_g, np.float64).reshape(N)
        ug = np.ascontiguousarray(u_g, np.float64).reshape(D * N)
        ul = np.ascontiguousarray(u_l, np.float64).reshape(D * N)
        pk = np.ascontiguousarray(p_k, np.float64).reshape(N)
        _load().orc_init(self._h, _dptr(a), _dptr(ug), _dptr(ul), _dptr(pk))

    def step(self, n=1):
        _load().orc_step(self._h, int(n))

    def moments(self):
        N, D = self.N, self.D
        out = dict(alpha_g=np.empty(N), u_g=np.empty((D, N)), u_l=np.empty((D, N)),
                   p_k=np.empty(N), S_g=np.empty(N), S_l=np.empty(N))
        _load().orc_moments(self._h, *[_dptr(out[k]) for k in ("alpha_g", "u_g", "u_l", "p_k", "S_g", "S_l")])
        return out

    def pops(self, s):
        """Populations of scheme s (0 g, 1 l, 2 alpha_g, 3 alpha_l, 4 beta_g, 5 beta_l), shape (Q, N)."""
        out = np.empty((self.Q, self.N))
        _load().orc_get_pops(self._h, int(s), _dptr(out))
        return out

    def set_pops(self, s, arr):
        a = np.ascontiguousarray(arr, np.float64).reshape(self.Q * self.N)
        _load().orc_set_pops(self._h, int(s), _dptr(a))

    def held(self):
        a, b, c = np.empty(self.N), np.empty(self.N), np.empty(self.N)
        _load().orc_get_held(self._h, _dptr(a), _dptr(b), _dptr(c))
        return dict(Spp_g=a, Spp_l=b, Lam=c)

    def equilibria(self, phi, eps, u, alpha, psi, S, G):
        """(f_I^eq(phi, eps, u), f^eq(alpha, u), f_L^eq(psi, S, G)) in this oracle's q order."""
        u = np.ascontiguousarray(u, np.float64)
        G = np.ascontiguousarray(G, np.float64)
        fI, fS, fL = np.empty(self.Q), np.empty(self.Q), np.empty(self.Q)
        _load().orc_equilibria(self._h, phi, eps, _dptr(u), alpha, psi, S, _dptr(G), _dptr(fI), _dptr(fS), _dptr(fL))
        return fI, fS, fL

    def diag(self):
        out = np.empty(8)
        _load().orc_diag(self._h, _dptr(out))
        return out
