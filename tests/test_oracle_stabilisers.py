"""Pins of the oracle's large-density-ratio stabilisers (Sec. 3.2) against
what the mathematics fixes on a homogeneous state.

On a periodic lattice whose fields are uniform, every gradient vanishes:
the beta populations that stream in all carry the same c, so
beta = sum_q f^eq(1, c) = 1 and S = 1 - beta = 0 (Sec. 2.3); grad(alpha) = 0,
so the stress term of Eqs. (Gg), (Gl) drops; with kappa_I = kappa_W = 0 and
g_hat = 0 there is no drag and no buoyancy.  What is left of one step is
(zeroth and first moments of Eqs. (lbmg), (lbml): the BGK term conserves both,
the forcing operator of Eq. (forcingoperator) adds S'' and G):

    eps_g <- eps_g + S''_g,    u_g <- u_g + S''_g u_g,
    eps_l <- eps_l + S''_l,    u_l <- u_l + S''_l u_l,

with the latched sources of Eq. (lbm-cont-1D-update): at t = r n_gamma

    S''_g = S_g - gamma |u_g|^2 (eps_g - 1)          Eq. (lbm-cont-g1Dhat)
    S''_l = S_l - gamma |u_l|^2 (phi eps_l - 1)       Eq. (lbm-cont-l1Dhat), third strategy,
          = - gamma |u_l|^2 (eps_g - 1)/R             phi of Eq. (lbm-phi-l)

and S'' held in between.  The recurrence below is written from those
equations alone; the oracle's full six-scheme step must follow it.

One term of the full step is not in the recurrence: the forcing changes u
every step while the alpha populations relax towards equilibrium with the
previous u, so their first moment J lags a u, which Eq. (gradlnalpha) reads
as a gradient of alpha; the stress term sigma . grad(alpha)/alpha of Eq.
(Gg) then adds ~3e-11 of u per step (u drifts ~2e-9 relative from the
recurrence over the 60 steps).  Hence the bars: the pressure deviations
eps - 1 within 1e-7 relative, u within 1e-8.  A sign flip of the dashpot
(growth instead of decay), the first or second strategy for the liquid, S
instead of S'' in the momentum, no latch, or a latch on another phase of t
each moves eps - 1 or u by 5e-6 to 4 relative
(test_recurrence_distinguishes_the_readings), far outside those bars.
"""
import numpy as np
import pytest

import oracle

PER = 0
CS2 = 1.0 / 3.0


def recurrence(eps_g, eps_l, ug, ul, R, gamma, n_gamma, steps):
    """Per-step (eps_g, eps_l, u_g, u_l, S''_g, S''_l) of the homogeneous state
    (float64, the equations of the module docstring)."""
    ug, ul = np.array(ug, float), np.array(ul, float)
    out = []
    Sg = Sl = 0.0
    for t in range(steps):
        if t % n_gamma == 0:
            Sg = 0.0 - gamma * float(ug @ ug) * (eps_g - 1.0)
            Sl = 0.0 - gamma * float(ul @ ul) * (eps_g - 1.0) / R
        eps_g, eps_l = eps_g + Sg, eps_l + Sl
        ug, ul = ug + Sg * ug, ul + Sl * ul
        out.append((eps_g, eps_l, ug.copy(), ul.copy(), Sg, Sl))
    return out


def _params(R, gamma, n_gamma, D):
    return dict(R=R, omega_g=0.8, omega_l=1.3, omega_alpha=1.5, drag_model=0, kappa_I=0.0, kappa_W=0.0,
                g_hat=0.0, g_axis=0, gamma=gamma, n_gamma=n_gamma, spalding_mode=2, alpha_floor=1e-8,
                bc_lo=(PER, PER, PER), bc_hi=(PER, PER, PER))


@pytest.mark.parametrize("lat,dims", [("D1Q3", (6, 1, 1)), ("D2Q9", (4, 3, 1)), ("D3Q19", (3, 3, 2))])
@pytest.mark.parametrize("n_gamma", [1, 7])
def test_dashpot_and_latch_follow_the_recurrence(lat, dims, n_gamma):
    D = {"D1Q3": 1, "D2Q9": 2, "D3Q19": 3}[lat]
    R, gamma, steps = 5.0, 1.0, 60
    ug0 = np.array([0.05, -0.03, 0.02])[:D]
    ul0 = np.array([-0.04, 0.025, 0.01])[:D]
    eps_g0 = 1.0 + 3e-3
    N = int(np.prod(dims))
    o = oracle.Oracle(lat, dims, _params(R, gamma, n_gamma, D))
    o.init(alpha_g=np.full(N, 0.3), u_g=np.repeat(ug0[:, None], N, 1), u_l=np.repeat(ul0[:, None], N, 1),
           p_k=np.full(N, CS2 * eps_g0))
    # eps_l = 1 at the initial state (its reading in the oracle's init)
    ref = recurrence(eps_g0, 1.0, ug0, ul0, R, gamma, n_gamma, steps)
    held_prev = None
    for t in range(steps):
        o.step(1)
        m = o.moments()
        eg, el, ug, ul, Sg, Sl = ref[t]
        assert np.allclose(m["p_k"] / CS2 - 1.0, eg - 1.0, rtol=1e-7, atol=0), (t, m["p_k"][0] / CS2, eg)
        assert np.allclose(o.pops(1).sum(axis=0) - 1.0, el - 1.0, rtol=1e-7, atol=0), t
        assert np.allclose(m["u_g"], ug[:, None], rtol=1e-8, atol=0), t
        assert np.allclose(m["u_l"], ul[:, None], rtol=1e-8, atol=0), t
        # the held sources are the latched values, which change only when
        # t = r n_gamma (the step just taken was step t)
        h = o.held()
        # (S = 1 - beta carries the rounding of sum_q f^eq(1, c) = 1, ~1e-16)
        assert np.allclose(h["Spp_g"], Sg, rtol=1e-7, atol=1e-14), t
        assert np.allclose(h["Spp_l"], Sl, rtol=1e-7, atol=1e-14), t
        if held_prev is not None and t % n_gamma != 0:
            assert np.array_equal(h["Spp_g"], held_prev["Spp_g"]), t
            assert np.array_equal(h["Spp_l"], held_prev["Spp_l"]), t
        held_prev = h
    # the dashpot damps the pressure deviation (a mechanical dashpot, Eq.
    # (lbm-cont-g1D-ohwada)): |eps_g - 1| decreased
    assert abs(ref[-1][0] - 1.0) < abs(eps_g0 - 1.0)


def test_recurrence_distinguishes_the_readings():
    """The pins above are discriminating: each alternative a plausible mistake
    would implement moves eps_g - 1, eps_l - 1 or u by at least 100 times the
    bars above after 60 steps."""
    R, gamma, n, steps = 5.0, 1.0, 7, 60
    ug, ul = np.array([0.05, -0.03]), np.array([-0.04, 0.025])
    base = recurrence(1.003, 1.0, ug, ul, R, gamma, n, steps)[-1]

    def variant(sign=1.0, liquid="third", phase=0, latch=True, s_in_g=True):
        eg, el, g, l = 1.003, 1.0, ug.copy(), ul.copy()
        Sg = Sl = 0.0
        for t in range(steps):
            if not latch or (t - phase) % n == 0:
                Sg = -sign * gamma * (g @ g) * (eg - 1.0)
                G = {"third": (eg - 1.0) / R, "first": el - 1.0, "second": eg - 1.0}[liquid]
                Sl = -sign * gamma * (l @ l) * G
            eg, el = eg + Sg, el + Sl
            if s_in_g:
                g, l = g + Sg * g, l + Sl * l
        return eg, el, g, l

    for kw in (dict(sign=-1.0), dict(liquid="first"), dict(liquid="second"), dict(phase=1), dict(latch=False),
               dict(s_in_g=False)):
        eg, el, g, l = variant(**kw)
        d_eps = max(abs(eg - base[0]) / abs(base[0] - 1.0), abs(el - base[1]) / abs(base[1] - 1.0))
        d_u = max(np.linalg.norm(g - base[2]) / np.linalg.norm(base[2]),
                  np.linalg.norm(l - base[3]) / np.linalg.norm(base[3]))
        assert d_eps > 100 * 1e-7 or d_u > 100 * 1e-8, kw
