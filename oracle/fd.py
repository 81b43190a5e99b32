"""Finite-difference reference solver of the 1D Eulerian-Eulerian system (Sec. 3.4).

TEST INFRASTRUCTURE (see oracle/__init__.py).  The paper validates its LBM
against a method-of-lines FD solution of the same target equations, in
lattice units:

  d p_k/dt  = -cs2 Dx u_g + cs2 Dx[alpha_l (u_g - u_l)]                     Eq. (lbm-cont-g1DFD)
  d u_g/dt  = -Dx(u_g u_g) - Dx p_k + nu_g Dx^2 u_g + S_g u_g
              + (sigma_g/alpha_g) Dx alpha_g + (R-1) g + (K_I/alpha_g)|u_l-u_g|(u_l-u_g)   Eq. (lbm-mom-g1DFD)
  d u_l/dt  = -Dx(u_l u_l) - (1/R) Dx p_k + nu_l Dx^2 u_l + S_l u_l
              + (sigma_l/alpha_l) Dx alpha_l + (1/R)(K_I/alpha_l)|u_g-u_l|(u_g-u_l)
              - (1/R)(K_W/alpha_l)|u_l| u_l                                  Eq. (lbm-mom-l1DFD)
  d alpha_g/dt = -Dx(alpha_g u_g)                                            Eq. (voidfraction1DFD)

with S_g = Dx[alpha_l (u_g - u_l)], S_l = Dx[alpha_g (u_l - u_g)] (Eqs.
(lbm-cont-g1D), (lbm-cont-l)), sigma = nu Dx u (Eq. (stresstensor1D)),
central differences Dx, Dx^2 (Eqs. (FD-Dx), (FD-DxDx)), K_I constant or
kappa_I Lambda(alpha_g) (Eq. (CliftGraceWeber)).  Reading: the wall-friction
term opposes u_l (its sign in Eq. (lbm-mom-l1DFD) is read as a typo, matching
Eq. (wallmomentum1D)); nu is the LBM's effective 1D viscosity (Eq.
(lbm-ef-viscosity)).  Periodic columns use wrap-around differences; walls use
ghost nodes u_0 = -u_1 (no flux through the half-way wall), alpha_0 = alpha_1,
p_k linear extrapolation.

Time integration: the Dormand-Prince 5(4) embedded Runge-Kutta pair with
adaptive steps (the method behind ode45), written from its published
coefficients; optional Gaussian moving-average smoothing of the solution every
`smooth_every` accepted steps (Sec. 3.4; window 12, sigma = window/5).

Parity: the solver's parts are pinned (the integrator on closed-form ODEs,
the right-hand side in the homogeneous limit and on single Fourier modes);
its agreement with the LBM is a cross-check at a tolerance, since the paper
reports that agreement only qualitatively.
"""
import numpy as np

CS2 = 1.0 / 3.0

# Dormand-Prince 5(4) coefficients (Dormand & Prince 1980)
_C = np.array([0.0, 1 / 5, 3 / 10, 4 / 5, 8 / 9, 1.0, 1.0])
_A = [
    [],
    [1 / 5],
    [3 / 40, 9 / 40],
    [44 / 45, -56 / 15, 32 / 9],
    [19372 / 6561, -25360 / 2187, 64448 / 6561, -212 / 729],
    [9017 / 3168, -355 / 33, 46732 / 5247, 49 / 176, -5103 / 18656],
    [35 / 384, 0.0, 500 / 1113, 125 / 192, -2187 / 6784, 11 / 84],
]
_B5 = np.array([35 / 384, 0.0, 500 / 1113, 125 / 192, -2187 / 6784, 11 / 84, 0.0])
_B4 = np.array([5179 / 57600, 0.0, 7571 / 16695, 393 / 640, -92097 / 339200, 187 / 2100, 1 / 40])


def dopri45(f, t0, y0, t1, rtol=1e-8, atol=1e-14, h0=None, max_steps=10 ** 8, callback=None):
    """Integrate y' = f(t, y) from t0 to t1 with the adaptive Dormand-Prince
    5(4) pair (local extrapolation, first-same-as-last).  `callback(n, t, y)`
    is called after every accepted step and may return a replacement y."""
    t, y = float(t0), np.array(y0, dtype=np.float64)
    k1 = f(t, y)
    h = h0 if h0 else min(1.0, abs(t1 - t0))
    n = 0
    while t < t1 and n < max_steps:
        h = min(h, t1 - t)
        k = [k1]
        for i in range(1, 7):
            yi = y + h * sum(_A[i][j] * k[j] for j in range(i))
            k.append(f(t + _C[i] * h, yi))
        y5 = y + h * sum(_B5[i] * k[i] for i in range(7) if _B5[i] != 0.0)
        y4 = y + h * sum(_B4[i] * k[i] for i in range(7) if _B4[i] != 0.0)
        sc = atol + rtol * np.maximum(np.abs(y), np.abs(y5))
        err = np.sqrt(np.mean(((y5 - y4) / sc) ** 2))
        if err <= 1.0:
            t += h
            y = y5
            k1 = k[6]
            n += 1
            if callback is not None:
                r = callback(n, t, y)
                if r is not None:
                    y = r
                    k1 = f(t, y)
        fac = 0.9 * (1.0 / err) ** 0.2 if err > 0 else 5.0
        h *= min(5.0, max(0.2, fac))
    return t, y, n


def gaussian_smooth(v, window=12, periodic=True):
    """Gaussian-weighted moving average (sigma = window/5)."""
    sigma = window / 5.0
    half = window // 2
    x = np.arange(-half, half + 1)
    w = np.exp(-0.5 * (x / sigma) ** 2)
    w /= w.sum()
    if periodic:
        return sum(w[i] * np.roll(v, -x[i]) for i in range(len(x)))
    pad = np.pad(v, half, mode="edge")
    return np.convolve(pad, w[::-1], mode="valid")


class FD1D:
    """State vector y = [p_k, u_g, u_l, alpha_g] (4 N values)."""

    def __init__(self, N, p, bc="periodic"):
        self.N = N
        self.p = dict(p)
        self.bc = bc
        om_g, om_l = p["omega_g"], p["omega_l"]
        # effective 1D viscosity of the LBM, Eq. (lbm-ef-viscosity)
        self.nu_g = (1.0 / om_g - 0.5) - CS2 * p.get("psi_g", 0.0) / om_g
        self.nu_l = (1.0 / om_l - 0.5) - CS2 * p.get("psi_l", 0.0) / om_l

    def _wrap(self, v, kind):
        """<v> with one ghost node each side."""
        if self.bc == "periodic":
            return np.concatenate([v[-1:], v, v[:1]])
        if kind == "u":          # no penetration half-way: u_0 = -u_1
            return np.concatenate([-v[:1], v, -v[-1:]])
        if kind == "a":          # zero gradient
            return np.concatenate([v[:1], v, v[-1:]])
        return np.concatenate([2 * v[:1] - v[1:2], v, 2 * v[-1:] - v[-2:-1]])  # p_k: linear extrapolation

    @staticmethod
    def Dx(w):
        return 0.5 * (w[2:] - w[:-2])                 # Eq. (FD-Dx)

    @staticmethod
    def Dxx(w):
        return w[2:] - 2.0 * w[1:-1] + w[:-2]         # Eq. (FD-DxDx)

    def rhs(self, t, y):
        N, p = self.N, self.p
        pk, ug, ul, ag = y[:N], y[N:2 * N], y[2 * N:3 * N], y[3 * N:]
        al = 1.0 - ag
        R, g = p["R"], p["g_hat"]
        Wpk, Wug, Wul, Wag = self._wrap(pk, "p"), self._wrap(ug, "u"), self._wrap(ul, "u"), self._wrap(ag, "a")
        Wal = 1.0 - Wag
        Sg = self.Dx(Wal * (Wug - Wul))
        Sl = self.Dx(Wag * (Wul - Wug))
        if p.get("drag_model", 0) == 1:
            lam = ag * al * (ag + al * R)
            KI, KW = p["kappa_I"] * lam, p.get("kappa_W", 0.0) * lam
        else:
            KI, KW = p["kappa_I"], p.get("kappa_W", 0.0)
        sg = self.nu_g * self.Dx(Wug)
        sl = self.nu_l * self.Dx(Wul)
        du = ul - ug
        dpk = -CS2 * self.Dx(Wug) + CS2 * Sg
        dug = (-self.Dx(Wug * Wug) - self.Dx(Wpk) + self.nu_g * self.Dxx(Wug) + Sg * ug
               + sg / ag * self.Dx(Wag) + (R - 1.0) * g + KI / ag * np.abs(du) * du)
        dul = (-self.Dx(Wul * Wul) - self.Dx(Wpk) / R + self.nu_l * self.Dxx(Wul) + Sl * ul
               + sl / al * self.Dx(Wal) + KI / (R * al) * np.abs(du) * (-du) - KW / (R * al) * np.abs(ul) * ul)
        dag = -self.Dx(Wag * Wug)
        return np.concatenate([dpk, dug, dul, dag])

    def run(self, fields, T, rtol=1e-8, smooth_every=0, window=12):
        N = self.N
        y0 = np.concatenate([fields["p_k"], fields["u_g"].reshape(-1), fields["u_l"].reshape(-1), fields["alpha_g"]])

        def cb(n, t, y):
            if smooth_every and n % smooth_every == 0:
                per = self.bc == "periodic"
                return np.concatenate([gaussian_smooth(y[k * N:(k + 1) * N], window, per) for k in range(4)])
            return None

        _, y, n = dopri45(self.rhs, 0.0, y0, float(T), rtol=rtol, callback=cb)
        return dict(p_k=y[:N], u_g=y[N:2 * N][None, :], u_l=y[2 * N:3 * N][None, :], alpha_g=y[3 * N:], steps=n)
