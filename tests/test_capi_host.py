"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports every
function include/lbm.h declares, and its host-only entry points (defaults,
velocity sets) agree with the oracle's independent lattice construction.
No GPU compute is called here."""
import ctypes
import os
import re

import numpy as np
import pytest

import lbm_inputs
import oracle
import paper_2409_10399_gb300 as lbm
from oracle import params as oparams
from paper_2409_10399_gb300 import params as lparams

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = lbm.load_library()
    names = header_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_params_struct_layout_matches_header_defaults():
    p = lbm.default_params()
    assert p.R == 2.0 and p.omega_g == 1.0 and p.omega_alpha == 1.5 and p.n_gamma == 1
    assert p.spalding_mode == 2 and p.alpha_floor == 1e-8 and p.precision == 1
    assert list(p.bc_lo) == [0, 0, 0] and p.diag_every == 0


@pytest.mark.parametrize("lat", ["D1Q3", "D2Q9", "D3Q19"])
def test_lattice_tables_match_oracle(lat):
    v, w = lbm.lattice_tables(lat)
    o = oracle.Oracle(lat, (2, 2 if lat != "D1Q3" else 1, 2 if lat == "D3Q19" else 1), {})
    vo, wo, _ = o.lattice_tables()
    mine = {tuple(r): x for r, x in zip(v.tolist(), w)}
    ref = {tuple(r): x for r, x in zip(vo.tolist(), wo)}
    assert mine == ref
    assert np.all(v[0] == 0)
    # lexicographic order of the moving velocities, so opp(q) = Q - q
    Q = len(w)
    for q in range(1, Q):
        assert np.all(v[q] == -v[Q - q])
    assert [tuple(r) for r in v[1:].tolist()] == sorted(tuple(r) for r in v[1:].tolist())
    # same order as the oracle's own construction (bitwise FP64 parity sums moments in this order)
    assert np.array_equal(v, vo) and np.array_equal(w, wo)


def test_invalid_lattice_rejected_without_gpu():
    lib = lbm.load_library()
    Q = ctypes.c_int()
    assert lib.lbm_lattice(4, ctypes.byref(Q), None, None) == -1


@pytest.mark.parametrize("name", ["column1d", "box2d", "column3d"])
def test_parameter_helpers_agree(name):
    ph = lbm_inputs.WORKLOADS[name]["physics"]
    a = oparams.lattice_params(ph)
    b = lparams.lattice_params(ph)
    for k, v in a.items():
        assert k in b
        if isinstance(v, float):
            assert b[k] == pytest.approx(v, rel=1e-14, abs=0), k
        else:
            assert tuple(np.atleast_1d(b[k])) == tuple(np.atleast_1d(v)), k


def test_tile_limit_matches_launch_bounds():
    """lbm_tile_limit reports the block size each fused step kernel is built
    for (host only): 128 for the D2Q9/D1Q3/D3Q19 float and half stores, 256
    for the double forms; unknown codes are rejected."""
    import paper_2409_10399_gb300 as lbm
    for lat in ("D1Q3", "D2Q9", "D3Q19"):
        assert lbm.tile_limit(lat, "fp32") == 128
        assert lbm.tile_limit(lat, "fp16dev") == 128
        assert lbm.tile_limit(lat, "fp64dev") == 256
        assert lbm.tile_limit(lat, "fp64") == 256
    with pytest.raises(lbm.LBMError):
        lbm.tile_limit(4, "fp32")
    with pytest.raises(lbm.LBMError):
        lbm.tile_limit("D2Q9", 7)


def test_surrogate_create_rejects_invalid_shapes_without_gpu():
    """lbm_fno_create validates its shape before touching the device: sizes
    not multiples of 16, channels not multiples of 16, modes not multiples of
    8 or above n / 2, and layer counts outside 1..16 give LBM_EINVAL; NULL
    handles are rejected by every surrogate entry point."""
    lib = lbm.load_library()
    h = ctypes.c_void_p()
    for args in [(24, 32, 16, 8, 1), (32, 40, 16, 8, 1), (32, 32, 24, 8, 1), (32, 32, 16, 12, 1),
                 (32, 32, 16, 24, 1), (32, 32, 16, 8, 0), (32, 32, 16, 8, 17), (8, 32, 16, 8, 1)]:
        assert lib.lbm_fno_create(*args, ctypes.byref(h)) == -1, args
        assert not h.value
    assert lib.lbm_fno_create(32, 32, 16, 8, 1, None) == -1
    assert lib.lbm_fno_set_loss(None, ctypes.c_double(1.0)) == -1
    assert lib.lbm_fno_set_inflow(None, ctypes.c_double(1.0)) == -1
    assert lib.lbm_fno_advance(None, None, None, ctypes.c_double(1e-4), None, None) == -1
    assert lib.lbm_surrogate_advance(None, None, 64, ctypes.c_double(1e-4), None, None) == -1
    assert lib.lbm_fno_destroy(None) == 0
    # the product alone: shapes are checked before any device access (the
    # addresses below are never dereferenced); empty or ragged (not a
    # multiple of 16) sizes, leading dimensions not multiples of 8, a split
    # K without beta = 1 are all LBM_EINVAL
    a = ctypes.c_void_p(1 << 20)
    f1, f0 = ctypes.c_float(1.0), ctypes.c_float(0.0)
    for (M, N, K, lda, beta, ks) in [(0, 16, 16, 16, f0, 1), (16, 0, 16, 16, f0, 1), (16, 16, 0, 16, f0, 1),
                                     (16, 16, 40, 48, f0, 1), (16, 16, 16, 12, f0, 1), (16, 16, 64, 64, f0, 2)]:
        assert lib.lbm_fno_gemm(0, 0, M, N, K, f1, a, lda, 0, a, 16, 0, beta, a, 16, 0, 1, 1, ks, None) == -1, \
            (M, N, K, lda, ks)


def _set(p, **kv):
    for k, v in kv.items():
        if k in ("bc_lo", "bc_hi", "in_alpha", "in_ug", "in_ul"):
            getattr(p, k)[:] = v
        else:
            setattr(p, k, v)
    return p


@pytest.mark.parametrize("bad", [
    dict(R=0.5), dict(omega_g=0.0), dict(omega_g=2.0), dict(omega_l=2.5), dict(omega_alpha=0.0),
    dict(n_gamma=0), dict(spalding_mode=3), dict(spalding_mode=-1), dict(alpha_floor=0.0), dict(g_axis=2),
    dict(g_axis=-1), dict(precision=5), dict(drag_model=2), dict(diag_every=-1), dict(beta_stencil=2),
    dict(beta_stencil=1, precision=0), dict(R=float("nan")), dict(omega_g=float("nan")),
    dict(bc_lo=[4, 1, 0], bc_hi=[4, 1, 0]),                      # unknown boundary code
    dict(bc_lo=[0, 1, 0], bc_hi=[1, 1, 0]),                      # periodic on one face only
    dict(bc_lo=[0, 1, 0], bc_hi=[0, 2, 0]),                      # inlet on the upper face
    dict(bc_lo=[0, 3, 0], bc_hi=[0, 1, 0]),                      # outlet on the lower face
    dict(bc_lo=[2, 1, 0], bc_hi=[1, 1, 0]),                      # inlet off the gravity axis
    dict(bc_lo=[0, 2, 0], bc_hi=[0, 1, 0], inlet_ul_mode=1, in_alpha=[1.0, 1.0]),  # no liquid to balance
])
def test_create_rejects_invalid_parameters_without_gpu(bad):
    """lbm_create checks every parameter before touching the device: each of
    these single faults gives LBM_EINVAL and leaves the handle NULL (the
    same parameters without the fault pass the checks: without a GPU they
    fail only at the device allocation, LBM_ENOMEM)."""
    lib = lbm.load_library()
    ok = _set(lbm.default_params(), g_axis=1, bc_lo=[0, 1, 0], bc_hi=[0, 1, 0])
    h0 = ctypes.c_void_p()
    rc = lib.lbm_create(2, 2, 64, 32, 1, ctypes.byref(ok), ctypes.byref(h0))
    assert rc in (0, -2), rc
    if rc == 0:
        lib.lbm_destroy(h0)
    p = _set(lbm.default_params(), **dict(dict(g_axis=1, bc_lo=[0, 1, 0], bc_hi=[0, 1, 0]), **bad))
    h = ctypes.c_void_p(12345)
    assert lib.lbm_create(2, 2, 64, 32, 1, ctypes.byref(p), ctypes.byref(h)) == -1, bad
    assert not h.value


@pytest.mark.parametrize("dims", [(3, 2, 64, 32, 1), (2, 2, 64, 32, 2), (1, 1, 64, 2, 1), (2, 2, 0, 32, 1),
                                  (2, 2, 1 << 16, 1 << 15, 1), (4, 4, 8, 8, 8)])
def test_create_rejects_invalid_shapes_without_gpu(dims):
    lib = lbm.load_library()
    p = _set(lbm.default_params(), g_axis=0)
    h = ctypes.c_void_p(12345)
    assert lib.lbm_create(*dims, ctypes.byref(p), ctypes.byref(h)) == -1, dims
    assert not h.value
    assert lib.lbm_create(2, 2, 64, 32, 1, None, ctypes.byref(h)) == -1
    assert lib.lbm_create(2, 2, 64, 32, 1, ctypes.byref(p), None) == -1


def test_batch_create_rejects_invalid_without_gpu():
    """lbm_batch_create's checks that come before any device access: lattice
    code, instance count, NULL arrays, the FP64 reference form (the batched
    kernel runs the deviation forms), and an instance with an inlet, an
    outlet or the beta-stencil form (the batched kernel has neither)."""
    lib = lbm.load_library()
    h = ctypes.c_void_p(12345)
    dims = (ctypes.c_int * 3)(64, 32, 1)
    base = dict(g_axis=1, bc_lo=[0, 1, 0], bc_hi=[0, 1, 0])
    for lat, n, d, kv in [(4, 1, dims, {}), (2, 0, dims, {}), (2, 1, None, {}), (2, 1, dims, dict(precision=0)),
                          (2, 1, dims, dict(bc_lo=[0, 2, 0])), (2, 1, dims, dict(bc_hi=[0, 3, 0])),
                          (2, 1, dims, dict(beta_stencil=1))]:
        p = _set(lbm.default_params(), **dict(base, **kv))
        assert lib.lbm_batch_create(lat, n, d, ctypes.byref(p), ctypes.byref(h)) == -1, (lat, n, kv)
        assert not h.value
    assert lib.lbm_batch_create(2, 1, dims, None, ctypes.byref(h)) == -1
    assert lib.lbm_batch_destroy(None) == 0


def test_every_entry_point_rejects_null_handles():
    """Every function include/lbm.h declares, called with NULL handles and
    pointers and zero sizes (no GPU): LBM_EINVAL, except the NULL-safe
    destroys (LBM_OK), the error-message accessors ("") and
    lbm_default_params (nothing to fill)."""
    lib = lbm.load_library()
    for name in header_functions():
        fn = getattr(lib, name)
        assert fn.argtypes is not None, name  # every declared function has its signature in the binding
        args = []
        for t in fn.argtypes:
            if t in (ctypes.c_int, ctypes.c_longlong, ctypes.c_uint):
                args.append(0)
            elif t in (ctypes.c_double, ctypes.c_float):
                args.append(0.0)
            else:
                args.append(None)
        rc = fn(*args)
        if name.endswith("_destroy"):
            assert rc == 0, name
        elif name.endswith("last_error"):
            assert rc in (b"", None), name
        elif name == "lbm_default_params":
            assert rc is None
        else:
            assert rc == -1, (name, rc)
