"""The paper's own validation (Sec. 3.4, 3.6): the LBM against an independent
finite-difference solution of the same 1D Eulerian-Eulerian equations.

* The FD solver's integrator (Dormand-Prince 5(4), the pair behind ode45) is
  pinned on ODEs with closed-form solutions.
* The FD right-hand side reduces, for a uniform state, to the 0-D momentum
  balance of Sec. 3.1 (buoyancy, drag, wall friction).
* On a smooth periodic column (TEST #1 physics, sinusoidal alpha_g) the
  oracle LBM and the FD solution agree; the paper reports this agreement only
  qualitatively ("excellent"), so the bars are set from the O(eps^2)
  truncation of both schemes at 128 nodes per wavelength (parity: partial).
"""
import numpy as np
import pytest

import oracle
from oracle import fd


def test_dopri45_exponential_and_oscillator():
    t, y, n = fd.dopri45(lambda t, y: -y, 0.0, np.array([1.0]), 5.0, rtol=1e-10, atol=1e-14)
    assert t == pytest.approx(5.0) and abs(y[0] - np.exp(-5.0)) < 1e-11
    f = lambda t, y: np.array([y[1], -y[0]])
    t, y, n = fd.dopri45(f, 0.0, np.array([1.0, 0.0]), 10.0, rtol=1e-10, atol=1e-14)
    assert abs(y[0] - np.cos(10.0)) < 1e-8 and abs(y[1] + np.sin(10.0)) < 1e-8
    # tighter tolerance -> smaller error (the controller works)
    e = [abs(fd.dopri45(lambda t, y: -y, 0.0, np.array([1.0]), 5.0, rtol=r, atol=1e-16)[1][0] - np.exp(-5.0))
         for r in (1e-5, 1e-9)]
    assert e[1] < e[0] * 1e-2


def test_fd_rhs_homogeneous_limit():
    N = 8
    p = dict(R=2.0, omega_g=0.6, omega_l=0.9, kappa_I=1e-2, kappa_W=2e-2, g_hat=1e-6, drag_model=0)
    s = fd.FD1D(N, p)
    ag, ug, ul = 0.3, 2e-3, 5e-4
    y = np.concatenate([np.full(N, 1 / 3), np.full(N, ug), np.full(N, ul), np.full(N, ag)])
    r = s.rhs(0.0, y)
    du = ul - ug
    assert np.allclose(r[:N], 0.0, atol=1e-20)
    assert np.allclose(r[N:2 * N], (2.0 - 1.0) * 1e-6 + 1e-2 / ag * abs(du) * du, rtol=1e-12)
    assert np.allclose(r[2 * N:3 * N], 1e-2 / (2.0 * 0.7) * abs(du) * (-du) - 2e-2 / (2.0 * 0.7) * abs(ul) * ul,
                       rtol=1e-12)
    assert np.allclose(r[3 * N:], 0.0, atol=1e-20)


@pytest.mark.parametrize("T,bars", [(2000, (1e-3, 2e-3, 1e-2, 1e-2)), (8000, (2e-3, 2e-3, 5e-3, 1e-2))])
def test_lbm_agrees_with_fd(T, bars):
    N = 128
    p = dict(R=2.0, omega_g=0.6, omega_l=0.6, omega_alpha=1.999, drag_model=0, kappa_I=1e-2, kappa_W=1e-2,
             g_hat=1e-6, g_axis=0, gamma=0.0, n_gamma=1, spalding_mode=2)
    x = np.arange(N)
    f = dict(alpha_g=0.3 + 0.1 * np.sin(2 * np.pi * x / N), u_g=np.zeros((1, N)), u_l=np.zeros((1, N)),
             p_k=np.full(N, 1 / 3))
    o = oracle.Oracle("D1Q3", (N, 1, 1), p)
    o.init(**f)
    o.step(T)
    m = o.moments()
    ref = fd.FD1D(N, p).run(f, T, rtol=1e-9)
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(m["alpha_g"], ref["alpha_g"]) < bars[0]
    assert rel(m["u_g"], ref["u_g"]) < bars[1]
    assert rel(m["u_l"], ref["u_l"]) < bars[2]
    assert rel(m["p_k"] - 1 / 3, ref["p_k"] - 1 / 3) < bars[3]
