"""The paper's own validation (Sec. 3.4, 3.6): the LBM against an independent
finite-difference solution of the same 1D Eulerian-Eulerian equations.

* The FD solver's integrator (Dormand-Prince 5(4), the pair behind ode45) is
  pinned on ODEs with closed-form solutions.
* The FD right-hand side reduces, for a uniform state, to the 0-D momentum
  balance of Sec. 3.1 (buoyancy, drag, wall friction), and on single Fourier
  modes to closed forms through the central differences' symbols
  (advection, the gas continuity with its source, viscosity).
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


def test_fd_rhs_single_fourier_modes():
    """Single Fourier modes on a periodic column, where the central
    differences act through their symbols (Dx sin kx = sin k cos kx,
    Dxx sin kx = -2 (1 - cos k) sin kx) and the right-hand side has a closed
    form: (a) a volume-fraction wave carried by a uniform velocity of both
    phases is advected, nothing else moves (no slip: no source, no drag, no
    stress); (b) a gas velocity wave in a uniform mixture changes the
    pressure through the gas continuity with its source, -cs2 alpha_g Dx u_g
    (Eqs. (lbm-cont-g1DFD), (lbm-cont-g1D)), the gas momentum through
    advection, viscosity and the source term S_g u_g, and the volume
    fraction through -alpha_g Dx u_g."""
    N, m, eps = 64, 3, 1e-3
    k = 2 * np.pi * m / N
    x = np.arange(N)
    sn, cs = np.sin(k * x), np.cos(k * x)
    p = dict(R=5.0, omega_g=0.7, omega_l=1.1, kappa_I=0.0, kappa_W=0.0, g_hat=0.0, drag_model=0)
    s = fd.FD1D(N, p)
    nu_g = 1.0 / 0.7 - 0.5
    # (a) alpha_g = a0 + eps sin kx, u_g = u_l = U, p_k uniform
    a0, U = 0.3, 2e-3
    y = np.concatenate([np.full(N, 1 / 3), np.full(N, U), np.full(N, U), a0 + eps * sn])
    r = s.rhs(0.0, y)
    assert np.allclose(r[:N], 0.0, atol=1e-18)
    assert np.allclose(r[N:3 * N], 0.0, atol=1e-18)
    assert np.allclose(r[3 * N:], -U * eps * np.sin(k) * cs, rtol=1e-12, atol=1e-18)
    # (b) u_g = eps sin kx, u_l = 0, alpha_g = a0, p_k uniform
    y = np.concatenate([np.full(N, 1 / 3), eps * sn, np.zeros(N), np.full(N, a0)])
    r = s.rhs(0.0, y)
    al = 1.0 - a0
    assert np.allclose(r[:N], -(1 / 3) * a0 * eps * np.sin(k) * cs, rtol=1e-12, atol=1e-20)
    s2 = np.sin(2 * k * x)
    want_ug = (-eps ** 2 * 0.5 * np.sin(2 * k) * s2          # -Dx(u_g^2), u_g^2 = eps^2 (1 - cos 2kx) / 2
               - 2.0 * nu_g * (1.0 - np.cos(k)) * eps * sn   # nu_g Dxx u_g
               + al * eps ** 2 * 0.5 * np.sin(k) * s2)       # S_g u_g, S_g = alpha_l eps sin k cos kx
    assert np.allclose(r[N:2 * N], want_ug, rtol=1e-10, atol=1e-16)
    # the liquid: its source S_l = Dx[alpha_g (u_l - u_g)] times u_l = 0, the pressure uniform, no drag
    assert np.allclose(r[2 * N:3 * N], 0.0, atol=1e-20)
    # the volume fraction carried by the gas wave, -Dx(alpha_g u_g) (Eq. (voidfraction1DFD))
    assert np.allclose(r[3 * N:], -a0 * eps * np.sin(k) * cs, rtol=1e-12, atol=1e-18)


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
