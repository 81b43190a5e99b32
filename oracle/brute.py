"""Independent brute-force stepper for tiny lattices (TEST INFRASTRUCTURE).

A second, deliberately different implementation of one EE-LBM time step
(arXiv 2409.10399, Sec. 2 and Sec. 3.2-3.5), in extended precision (mpmath,
40 digits), used to pin the C oracle on 3x4, 3x3x3 and 1D lattices for a few
steps.  Differences from lbm_oracle.c, on purpose:
  * the lattice is a dict {velocity tuple: weight}; D2Q9 is built as the
    tensor product of D1Q3, D3Q19 by listing the |v|^2 <= 2 subset of
    {-1,0,1}^3 with weights by speed;
  * populations are dicts keyed by (node tuple, velocity tuple);
  * tensor contractions are written as explicit double sums;
  * streaming is a pull from the neighbour (or the boundary rule).
Readings follow the same conventions as the C oracle (they are the paper's
readings, not implementation choices).
"""
import itertools

import mpmath as mp

mp.mp.dps = 40
CS2 = mp.mpf(1) / 3

PERIODIC, WALL, INLET, OUTLET = 0, 1, 2, 3
SCHEMES = ("g", "l", "ag", "al", "bg", "bl")


def lattice(D):
    w1 = {(0,): mp.mpf(2) / 3, (1,): mp.mpf(1) / 6, (-1,): mp.mpf(1) / 6}
    if D == 1:
        return w1
    if D == 2:
        return {(a[0], b[0]): wa * wb for a, wa in w1.items() for b, wb in w1.items()}
    out = {}
    for v in itertools.product((-1, 0, 1), repeat=3):
        s = sum(c * c for c in v)
        if s <= 2:
            out[v] = {0: mp.mpf(1) / 3, 1: mp.mpf(1) / 18, 2: mp.mpf(1) / 36}[s]
    return out


def rest(v):
    return all(c == 0 for c in v)


def contract(v, u):
    """(v v - cs2 I) : u u as an explicit double sum."""
    D = len(v)
    return sum((v[a] * v[b] - (CS2 if a == b else 0)) * u[a] * u[b] for a in range(D) for b in range(D))


def vdot(v, u):
    return sum(v[a] * u[a] for a in range(len(v)))


def eta(W, v, phi):
    w0 = W[tuple([0] * len(v))]
    return (1 + (1 - w0) / w0 * (1 - phi)) if rest(v) else phi


def fI(W, v, phi, eps, u):
    return W[v] * (eps * eta(W, v, phi) + vdot(v, u) / CS2 + contract(v, u) / (2 * CS2 ** 2))


def fS(W, v, alpha, u):
    return W[v] * alpha * (1 + vdot(v, u) / CS2 + contract(v, u) / (2 * CS2 ** 2))


def fL(W, v, psi, S, G):
    return W[v] * (S * eta(W, v, psi) + vdot(v, G) / CS2)


def ramp(mm, t, nt):
    if nt <= 0:
        return mp.mpf(mm[1])
    return (mp.mpf(mm[1]) - mp.mpf(mm[0])) * mp.tanh(mp.mpf(t) / nt) + mp.mpf(mm[0])


class Brute:
    def __init__(self, D, dims, p):
        self.D = D
        self.dims = tuple(dims[:D])
        self.W = lattice(D)
        self.V = sorted(self.W.keys())
        self.p = p
        self.nodes = list(itertools.product(*[range(n) for n in self.dims]))
        self.t = 0

    def idx(self, x):
        i, m = 0, 1
        for a in range(self.D):
            i += x[a] * m
            m *= self.dims[a]
        return i

    def init(self, alpha_g, u_g, u_l, p_k):
        W, D = self.W, self.D
        R = mp.mpf(self.p["R"])
        self.f = {s: {} for s in SCHEMES}
        self.Spp = {"g": {}, "l": {}}
        self.Lam = {}
        for x in self.nodes:
            i = self.idx(x)
            ag = mp.mpf(alpha_g[i])
            al = 1 - ag
            ug = [mp.mpf(u_g[a][i]) for a in range(D)]
            ul = [mp.mpf(u_l[a][i]) for a in range(D)]
            eg = mp.mpf(p_k[i]) / CS2
            el = mp.mpf(1)
            phi = (1 + (eg - 1) / R) / el
            cg = [al * (ug[a] - ul[a]) for a in range(D)]
            cl = [ag * (ul[a] - ug[a]) for a in range(D)]
            for v in self.V:
                self.f["g"][x, v] = fI(W, v, 1, eg, ug)
                self.f["l"][x, v] = fI(W, v, phi, el, ul)
                self.f["ag"][x, v] = fS(W, v, ag, ug)
                self.f["al"][x, v] = fS(W, v, al, ul)
                self.f["bg"][x, v] = fS(W, v, 1, cg)
                self.f["bl"][x, v] = fS(W, v, 1, cl)
            self.Spp["g"][x] = mp.mpf(0)
            self.Spp["l"][x] = mp.mpf(0)
            self.Lam[x] = ag * al * (ag + al * R)
        self.t = 0

    def _node(self, x, latch):
        p, W, D, V = self.p, self.W, self.D, self.V
        R = mp.mpf(p["R"])
        f = {s: [self.f[s][x, v] for v in V] for s in SCHEMES}
        mom0 = {s: sum(f[s]) for s in SCHEMES}
        mom1 = {s: [sum(V[k][a] * f[s][k] for k in range(len(V))) for a in range(D)] for s in ("g", "l", "ag", "al")}
        Pi = {s: [[sum(V[k][a] * V[k][b] * f[s][k] for k in range(len(V))) for b in range(D)] for a in range(D)]
              for s in ("g", "l")}
        eps = {"g": mom0["g"], "l": mom0["l"]}
        u = {"g": mom1["g"], "l": mom1["l"]}
        a_raw = {"g": mom0["ag"], "l": mom0["al"]}
        J = {"g": mom1["ag"], "l": mom1["al"]}
        S = {"g": 1 - mom0["bg"], "l": 1 - mom0["bl"]}
        mode = p["spalding_mode"]
        if mode == 0:
            alB = dict(a_raw)
        else:
            B = {k: min(max(a_raw[k], mp.mpf(0)), mp.mpf(1)) for k in ("g", "l")}
            tot = B["g"] + B["l"]
            g_ = B["g"] / tot if tot > 0 else mp.mpf(1) / 2
            alB = {"g": g_, "l": 1 - g_}
        phi = (1 + (eps["g"] - 1) / R) / eps["l"]
        phis = {"g": mp.mpf(1), "l": phi}
        gam = mp.mpf(p["gamma"])
        Sp = {"g": S["g"] - gam * vdot(u["g"], u["g"]) * (eps["g"] - 1),
              "l": S["l"] - gam * vdot(u["l"], u["l"]) * (phi * eps["l"] - 1)}
        if latch:
            self.Spp["g"][x] = Sp["g"]
            self.Spp["l"][x] = Sp["l"]
            self.Lam[x] = alB["g"] * alB["l"] * (alB["g"] + alB["l"] * R)
        Spp = {"g": self.Spp["g"][x], "l": self.Spp["l"][x]}
        Lam = self.Lam[x]
        oa = mp.mpf(p["omega_alpha"])
        grad = {k: [oa / CS2 * (a_raw[k] * u[k][a] - J[k][a]) for a in range(D)] for k in ("g", "l")}
        delta = [grad["g"][a] + grad["l"][a] for a in range(D)]
        gradG = {k: [grad[k][a] - delta[a] / 2 for a in range(D)] for k in ("g", "l")}
        om = {"g": mp.mpf(p["omega_g"]), "l": mp.mpf(p["omega_l"])}
        psi = {"g": mp.mpf(p["psi_g"]), "l": mp.mpf(p["psi_l"])}
        sig = {}
        for k in ("g", "l"):
            Peq = [[(CS2 * phis[k] * eps[k] if a == b else 0) + u[k][a] * u[k][b] for b in range(D)] for a in range(D)]
            if D == 1:
                nuef = (1 / om[k] - mp.mpf(1) / 2) - CS2 * psi[k] / om[k]
                sig[k] = [[nuef * (om[k] * (Peq[0][0] - Pi[k][0][0]) + psi[k] * CS2 * Spp[k])]]
            else:
                sig[k] = [[(1 - om[k] / 2) * (Peq[a][b] - Pi[k][a][b]) - (CS2 * psi[k] / 2 * Spp[k] if a == b else 0)
                           for b in range(D)] for a in range(D)]
        cgw = p["drag_model"] == 1
        KI = mp.mpf(p["kappa_I"]) * (Lam if cgw else 1)
        KW = mp.mpf(p["kappa_W"]) * (Lam if cgw else 1)
        floor = mp.mpf(p["alpha_floor"])
        den = {k: max(alB[k], floor) for k in ("g", "l")}
        du = [u["l"][a] - u["g"][a] for a in range(D)]
        ndu = mp.sqrt(vdot(du, du))
        nul = mp.sqrt(vdot(u["l"], u["l"]))
        buoy = (R - 1) * mp.mpf(p["g_hat"])
        G = {"g": [], "l": []}
        for a in range(D):
            sgrad_g = sum(sig["g"][a][b] * gradG["g"][b] for b in range(D))
            sgrad_l = sum(sig["l"][a][b] * gradG["l"][b] for b in range(D))
            G["g"].append(Spp["g"] * u["g"][a] + sgrad_g / den["g"] + (buoy if a == p["g_axis"] else 0)
                          + KI * ndu * du[a] / den["g"])
            G["l"].append(Spp["l"] * u["l"][a] + sgrad_l / den["l"] - KI * ndu * du[a] / (R * den["l"])
                          - KW * nul * u["l"][a] / (R * den["l"]))
        aeq = alB if mode == 2 else a_raw
        c = {"g": [alB["l"] * (u["g"][a] - u["l"][a]) for a in range(D)],
             "l": [alB["g"] * (u["l"][a] - u["g"][a]) for a in range(D)]}
        post = {s: {} for s in SCHEMES}
        for k, v in enumerate(V):
            post["g"][v] = f["g"][k] + om["g"] * (fI(W, v, 1, eps["g"], u["g"]) - f["g"][k]) + fL(W, v, psi["g"], Spp["g"], G["g"])
            post["l"][v] = f["l"][k] + om["l"] * (fI(W, v, phi, eps["l"], u["l"]) - f["l"][k]) + fL(W, v, psi["l"], Spp["l"], G["l"])
            post["ag"][v] = f["ag"][k] + oa * (fS(W, v, aeq["g"], u["g"]) - f["ag"][k])
            post["al"][v] = f["al"][k] + oa * (fS(W, v, aeq["l"], u["l"]) - f["al"][k])
            post["bg"][v] = fS(W, v, 1, c["g"])
            post["bl"][v] = fS(W, v, 1, c["l"])
        info = dict(eps=eps, u=u, alB=alB, c=c, phi=phi)
        return post, info

    def step(self, n=1):
        for _ in range(n):
            self._step1()

    def _step1(self):
        p, D, W = self.p, self.D, self.W
        latch = self.t % max(1, p["n_gamma"]) == 0
        post, info = {}, {}
        for x in self.nodes:
            post[x], info[x] = self._node(x, latch)
        ax = p["g_axis"]
        tr = next((d for d in range(D) if d != ax), None)
        R = mp.mpf(p["R"])
        new = {s: {} for s in SCHEMES}
        for x in self.nodes:
            for v in self.V:
                # pull: the population arriving at x with velocity v left x - v
                src = list(x)
                kinds = []
                for a in range(D):
                    src[a] -= v[a]
                    if src[a] < 0 or src[a] >= self.dims[a]:
                        bc = p["bc_lo"][a] if src[a] < 0 else p["bc_hi"][a]
                        if bc == PERIODIC:
                            src[a] %= self.dims[a]
                        else:
                            if bc == INLET and tr is not None and not (p["inlet_lo"] <= x[tr] < p["inlet_hi"]):
                                bc = WALL
                            kinds.append(bc)
                if not kinds:
                    for s in SCHEMES:
                        new[s][x, v] = post[tuple(src)][s][v]
                    continue
                kind = WALL if WALL in kinds else kinds[0]
                vo = tuple(-c for c in v)  # the population that left x towards the face
                for s in SCHEMES:
                    new[s][x, v] = self._bc(s, x, v, vo, kind, post, info)
        self.f = new
        self.t += 1

    def _nb(self, x, sign):
        y = list(x)
        y[self.p["g_axis"]] += sign
        return tuple(y)

    def _bc(self, s, x, vin, vout, kind, post, info):
        p, W, D = self.p, self.W, self.D
        R = mp.mpf(p["R"])
        fout = post[x][s][vout]
        if kind == WALL:
            return fout
        ax = p["g_axis"]
        if kind == INLET:
            y = self._nb(x, +1)
            aIN = ramp(p["in_alpha"], self.t, p["ramp_nt"])
            ugIN = ramp(p["in_ug"], self.t, p["ramp_nt"])
            ulIN = -aIN * ugIN / (1 - aIN) if p["inlet_ul_mode"] == 1 else ramp(p["in_ul"], self.t, p["ramp_nt"])
            e = [mp.mpf(1) if a == ax else mp.mpf(0) for a in range(D)]
            if s in ("g", "l"):
                ub = ugIN if s == "g" else ulIN
                uB = [ub * c for c in e]
                muB = [-c for c in uB]
                eg = mp.mpf(3) / 2 * info[x]["eps"]["g"] - info[y]["eps"]["g"] / 2
                el = mp.mpf(3) / 2 * info[x]["eps"]["l"] - info[y]["eps"]["l"] / 2
                if s == "g":
                    return fout + fI(W, vout, 1, eg, muB) - fI(W, vout, 1, eg, uB)
                ph = (1 + (eg - 1) / R) / el
                return fout + fI(W, vout, ph, el, muB) - fI(W, vout, ph, el, uB)
            if s in ("ag", "al"):
                ub = ugIN if s == "ag" else ulIN
                ab = aIN if s == "ag" else 1 - aIN
                return fS(W, vin, ab, [ub * c for c in e])
            k = "g" if s == "bg" else "l"
            cB = [2 * info[x]["c"][k][a] - info[y]["c"][k][a] for a in range(D)]
            return fS(W, vin, 2 * 1 - 1, cB)
        # OUTLET
        y = self._nb(x, -1)
        k = "g" if s in ("g", "ag", "bg") else "l"
        if s in ("g", "l", "ag", "al"):
            uB = [mp.mpf(3) / 2 * info[x]["u"][k][a] - info[y]["u"][k][a] / 2 for a in range(D)]
            muB = [-c for c in uB]
            if s in ("g", "l"):
                return -fout + fI(W, vout, 1, 1, muB) + fI(W, vout, 1, 1, uB)
            ab = mp.mpf(3) / 2 * info[x]["alB"][k] - info[y]["alB"][k] / 2
            return -fout + fS(W, vout, ab, muB) + fS(W, vout, ab, uB)
        cB = [2 * info[x]["c"][k][a] - info[y]["c"][k][a] for a in range(D)]
        return fS(W, vin, 2 * 1 - 1, cB)

    def pops(self, s):
        """Scheme s as {velocity tuple: [value per node in index order]}."""
        out = {}
        for v in self.V:
            col = [None] * len(self.nodes)
            for x in self.nodes:
                col[self.idx(x)] = self.f[s][x, v]
            out[v] = col
        return out
