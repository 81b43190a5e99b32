"""Pins of the oracle's lattices and equilibria against what the paper fixes.

* App. A, Eqs. (equilibriumD1Q3), (equilibriumID1Q3), (forcingoperatorD1Q3):
  the D1Q3 equilibria printed component by component must equal the oracle's
  general-D formulas (Eqs. (equilibrium), (equilibriumI), (forcingoperator)).
* Moment identities the paper states or uses: sum f_I^eq = eps, sum v f_I^eq = u
  (Sec. 2.1.1), second moment Eq. (secondtensoreq); moments of f^eq
  (Eq. (secondtensoreqalpha)); moments of the forcing operator (S, G, psi cs2 S I).
* Lattice isotropy up to fourth order, which the asymptotic analysis of
  Sec. 2.1.2 relies on (cs2 = 1/3).
"""
import itertools

import numpy as np
import pytest

import oracle

CS2 = 1.0 / 3.0


def _orc(lat):
    D = oracle.LATTICE_D[lat]
    dims = (2, 2 if D >= 2 else 1, 2 if D >= 3 else 1)
    return oracle.Oracle(lat, dims, {})


def test_lattice_sizes_and_opposites():
    for lat, Q in (("D1Q3", 3), ("D2Q9", 9), ("D3Q19", 19)):
        o = _orc(lat)
        v, w, opp = o.lattice_tables()
        assert o.Q == Q and v.shape == (Q, o.D)
        assert np.all(v[0] == 0), "rest velocity must be index 0 (delta_q, Eq. (delta))"
        assert np.all(v[opp] == -v)
        assert len({tuple(r) for r in v}) == Q


@pytest.mark.parametrize("lat", ["D1Q3", "D2Q9", "D3Q19"])
def test_lattice_isotropy(lat):
    o = _orc(lat)
    v, w, _ = o.lattice_tables()
    D = o.D
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(np.einsum("q,qa->a", w, v), 0.0, atol=1e-16)
    M2 = np.einsum("q,qa,qb->ab", w, v, v)
    assert np.allclose(M2, CS2 * np.eye(D), atol=1e-15)
    M3 = np.einsum("q,qa,qb,qc->abc", w, v, v, v)
    assert np.allclose(M3, 0.0, atol=1e-16)
    M4 = np.einsum("q,qa,qb,qc,qd->abcd", w, v, v, v, v)
    I = np.eye(D)
    iso = CS2 ** 2 * (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I) + np.einsum("ad,bc->abcd", I, I))
    if D == 1:
        # D1Q3: sum w v^4 = 1/3 = 3 cs2^2, the 1D projection of the same identity
        assert abs(M4[0, 0, 0, 0] - 3 * CS2 ** 2) < 1e-15
    else:
        assert np.allclose(M4, iso, atol=1e-15)


def test_d1q3_appendix_A():
    """App. A: the printed D1Q3 equilibria, with v = (0, 1, -1)."""
    o = _orc("D1Q3")
    v, w, _ = o.lattice_tables()
    order = [int(np.where(v[:, 0] == c)[0][0]) for c in (0, 1, -1)]
    r = np.random.default_rng(11)
    for _ in range(50):
        phi, eps, u, alpha, psi, S, G = r.uniform(0.5, 1.5), r.uniform(0.9, 1.1), r.uniform(-0.1, 0.1), \
            r.uniform(0, 1), r.uniform(-1, 1), r.uniform(-1e-2, 1e-2), r.uniform(-1e-3, 1e-3)
        fI, fS, fL = o.equilibria(phi, eps, [u, 0, 0], alpha, psi, S, [G, 0, 0])
        fI, fS, fL = fI[order], fS[order], fL[order]
        eS = [alpha * (2.0 / 3.0 - u * u), alpha * (1 + 3 * u + 3 * u * u) / 6, alpha * (1 - 3 * u + 3 * u * u) / 6]
        eI = [eps * (3 - phi) / 3 - u * u, (eps * phi + 3 * u + 3 * u * u) / 6, (eps * phi - 3 * u + 3 * u * u) / 6]
        eL = [S * (3 - psi) / 3, (S * psi + 3 * G) / 6, (S * psi - 3 * G) / 6]
        assert np.allclose(fS, eS, rtol=1e-14, atol=1e-17)
        assert np.allclose(fI, eI, rtol=1e-14, atol=1e-17)
        assert np.allclose(fL, eL, rtol=1e-14, atol=1e-19)


@pytest.mark.parametrize("lat", ["D1Q3", "D2Q9", "D3Q19"])
def test_equilibrium_moments(lat):
    o = _orc(lat)
    v, w, _ = o.lattice_tables()
    D = o.D
    I = np.eye(D)
    r = np.random.default_rng(5 + D)
    for _ in range(20):
        phi, eps, alpha, psi = r.uniform(0.5, 1.5), r.uniform(0.9, 1.1), r.uniform(0, 1), r.uniform(-1, 1)
        S = r.uniform(-1e-2, 1e-2)
        u = r.uniform(-0.05, 0.05, D)
        G = r.uniform(-1e-3, 1e-3, D)
        fI, fS, fL = o.equilibria(phi, eps, np.r_[u, np.zeros(3 - D)], alpha, psi, S, np.r_[G, np.zeros(3 - D)])
        # f_I^eq: sum = eps, first moment = u (incompressible), second = phi cs2 eps I + u u
        assert abs(fI.sum() - eps) < 1e-15
        assert np.allclose(v.T @ fI, u, atol=1e-16)
        Pi = np.einsum("qa,qb,q->ab", v, v, fI)
        assert np.allclose(Pi, phi * CS2 * eps * I + np.outer(u, u), atol=1e-15)
        # third moment of f_I^eq, Eq. (thirdtensoreq-th): cs2 (u_i d_jk + u_j d_ik + u_k d_ij)
        if D >= 2:
            Phi = np.einsum("qa,qb,qc,q->abc", v, v, v, fI)
            ref = CS2 * (np.einsum("a,bc->abc", u, I) + np.einsum("b,ac->abc", u, I) + np.einsum("c,ab->abc", u, I))
            assert np.allclose(Phi, ref, atol=1e-16)
        # f^eq(alpha, u): sum = alpha, first = alpha u, second = cs2 alpha I + alpha u u
        assert abs(fS.sum() - alpha) < 1e-15
        assert np.allclose(v.T @ fS, alpha * u, atol=1e-16)
        assert np.allclose(np.einsum("qa,qb,q->ab", v, v, fS), CS2 * alpha * I + alpha * np.outer(u, u), atol=1e-15)
        # forcing operator: sum = S, first = G, second = psi cs2 S I
        assert abs(fL.sum() - S) < 1e-17
        assert np.allclose(v.T @ fL, G, atol=1e-18)
        assert np.allclose(np.einsum("qa,qb,q->ab", v, v, fL), psi * CS2 * S * I, atol=1e-17)
