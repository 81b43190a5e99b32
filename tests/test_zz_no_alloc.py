"""The allocation-free diagnostics entry point, through the C ABI.

lbm_diag_populations_noalloc serves callers that may not allocate device
memory (their own pool, or code where the CUDA allocator must not run): it
reduces a caller-owned population buffer with a fixed __device__ scratch
array.  It must agree with lbm_get_diag on the same state, call after call.
This file is collected last so that a stop-at-first-failure run has already
run every other test.
"""
import numpy as np
import pytest

import lbm_inputs
import paper_2409_10399_gb300 as lbm

pytestmark = pytest.mark.gpu


def _state(lat, dims, prec, steps, spalding=2, nan_node=None):
    torch = pytest.importorskip("torch")
    D = lbm.LATTICE[lat]
    p = dict(R=1000.0, omega_g=0.6, omega_l=120.0 / 67.0, omega_alpha=1.5, drag_model=1, kappa_I=2.4e-4,
             g_hat=1e-6 / 999.0, g_axis=D - 1, gamma=1.0, n_gamma=7, spalding_mode=spalding, precision=prec,
             bc_lo=(0, 1, 1)[:D] + (0,) * (3 - D), bc_hi=(0, 1, 1)[:D] + (0,) * (3 - D))
    s = lbm.Simulation(lat, dims, p)
    f = lbm_inputs.fields_random(D, dims, seed=12, alpha=(0.05, 0.6), u_amp=2e-3, pk_amp=1e-5)
    if nan_node is not None:
        f["u_g"][0, nan_node] = np.nan  # planted on the host, as a caller's bad input would be
    s.init(**f)
    s.step(steps)
    Q = {1: 3, 2: 9, 3: 19}[D]
    pops = torch.empty((6, Q, s.N), dtype=torch.float64, device="cuda")
    for sch in range(6):
        s._check(s._lib.lbm_get_populations(s._h, sch, lbm.ctypes.c_void_p(pops[sch].data_ptr()), 1),
                 "lbm_get_populations")
    return s, pops


# 700 x 500 nodes needs more blocks than the scratch holds, so the partial pass
# strides over the nodes.  lbm_get_diag reduces per-node moments formed in the
# store's arithmetic type while this entry point reduces the FP64 populations,
# so the bar is the tests' bar for that type: 1e-12 for FP64 arithmetic,
# 1e-5 for FP32.
# Each Spalding mode (0 off, 1 and 2 the clamped renormalisation of Eq.
# (spalding)) is compared on a lattice built with that mode.
@pytest.mark.parametrize("spalding", [0, 1, 2])
@pytest.mark.parametrize("lat,dims,prec", [("D2Q9", (700, 500), "fp64dev"), ("D3Q19", (24, 20, 18), "fp64"),
                                           ("D1Q3", (300,), "fp64"), ("D2Q9", (130, 70), "fp32")])
def test_noalloc_matches_get_diag(lat, dims, prec, spalding):
    torch = pytest.importorskip("torch")
    s, pops = _state(lat, dims, prec, 33, spalding=spalding)
    ref = s.diag()
    tol = 1e-5 if prec == "fp32" else 1e-12
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):  # two calls in a row share the scratch array
        out_dev = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
        lbm.diag_populations_noalloc(lat, spalding, pops.data_ptr(), s.N, out_dev.data_ptr(), 1, stream)
        out_host = np.full(8, np.nan)
        lbm.diag_populations_noalloc(lat, spalding, pops.data_ptr(), s.N, out_host.ctypes.data, 0, stream)
        got_dev = out_dev.cpu().numpy()
        for got in (got_dev, out_host):
            for k in (0, 1, 2, 4):
                assert got[k] == pytest.approx(ref[k], rel=tol), k
            # sums of small per-node differences: on the scale of the node count
            for k in (6, 7):
                assert got[k] == pytest.approx(ref[k], rel=tol, abs=tol * 1e-3 * s.N), k
            # a_g + a_l - 1 is a small difference of O(1) sums (~1e-6 here): its
            # rounding is ~1e-16 (FP64) or ~1e-7 (FP32) per node before squaring
            assert got[3] == pytest.approx(ref[3], rel=1e-6 if tol < 1e-6 else 0.2, abs=1e-30)
            assert got[5] == ref[5] == 0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_counts_non_finite_nodes(prec):
    """A NaN velocity planted at one node of the initial fields spreads over a
    few steps; both entry points count the same nodes with a non-finite
    population (slot 5), call after call."""
    torch = pytest.importorskip("torch")
    s, pops = _state("D2Q9", (64, 40), prec, 3, nan_node=1000)
    ref = s.diag()
    assert ref[5] > 1
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        out = np.full(8, -1.0)
        lbm.diag_populations_noalloc("D2Q9", 2, pops.data_ptr(), s.N, out.ctypes.data, 0, stream)
        assert out[5] == ref[5]


def test_noalloc_rejects_bad_sizes():
    torch = pytest.importorskip("torch")
    buf = torch.zeros(6 * 9, dtype=torch.float64, device="cuda")
    out = np.zeros(8)
    for n in (0, -5, lbm.ctypes.c_longlong(2 ** 31).value):
        with pytest.raises(lbm.LBMError) as e:
            lbm.diag_populations_noalloc("D2Q9", 2, buf.data_ptr(), n, out.ctypes.data, 0)
        assert e.value.code == -1
