"""Pins of the oracle's quadrature against independent mathematics: exactness on
polynomials, and the analytic static potentials / singular pair rule against a
polar-coordinate brute force (Sec. II integrals)."""
import numpy as np
import pytest

from oracle.quadrature import (gauss_legendre01, map_rule, polar_integrate,
                               static_potentials, triangle_rule)

TRI = np.array([[0.0, 0.0, 0.0], [1.3, 0.2, 0.0], [0.3, 0.9, 0.1]])


def test_gauss_legendre_exactness():
    for n in range(1, 9):
        x, w = gauss_legendre01(n)
        for d in range(2 * n):
            assert abs(np.sum(w * x ** d) - 1.0 / (d + 1)) < 1e-14


def test_triangle_rule_exactness():
    # monomials on the reference triangle: int xi^a eta^b = a! b! / (a+b+2)!
    from math import factorial
    for n in range(1, 8):
        xi, eta, w = triangle_rule(n)
        for a in range(2 * n - 1):
            for b in range(2 * n - 1 - a):
                exact = factorial(a) * factorial(b) / factorial(a + b + 2)
                assert abs(np.sum(w * xi ** a * eta ** b) - exact) < 1e-15


def _ref_points():
    c = TRI.mean(0)
    n = np.cross(TRI[1] - TRI[0], TRI[2] - TRI[0])
    n /= np.linalg.norm(n)
    return [c, c + 0.3 * n, c + 1e-2 * n, 0.5 * (TRI[0] + TRI[1]), TRI[2],
            np.array([2.0, -1.0, 0.5]), TRI[0] + 0.2 * (TRI[0] - TRI[1])]


@pytest.mark.parametrize("i", range(7))
def test_static_potentials_vs_polar(i):
    r = _ref_points()[i]
    I1, Iv = static_potentials(r[None], TRI)
    n = np.cross(TRI[1] - TRI[0], TRI[2] - TRI[0])
    n /= np.linalg.norm(n)
    rho = r - ((r - TRI[0]) @ n) * n
    b1 = polar_integrate(r, TRI, lambda X, R: 1.0 / R, 48, 160, subdiv=6)
    bv = polar_integrate(r, TRI, lambda X, R: (X - rho) / R[:, None], 48, 160, subdiv=6)
    assert abs(I1[0] - b1) < 1e-11 * max(1, abs(b1))
    assert np.abs(Iv[0] - bv).max() < 1e-11


def test_singular_pair_rule_vs_bruteforce():
    """Close-pair rule (analytic static inner part + Gauss smooth remainder,
    symmetrized) against polar inner integration of the full kernel with a
    dense outer rule; coincident and edge-adjacent pairs."""
    import efie_inputs as E
    from oracle import dense
    from oracle.geometry import build_rwg
    V, T = E.icosphere(2, 0.5)
    m = build_rwg(V, T)
    k = 2 * np.pi
    # triangle 0, a neighbour sharing an edge, and a vertex neighbour
    t0 = 0
    shared = [t for t in range(m.Nt) if len(set(T[t]) & set(T[t0])) == 2][0]
    vert = [t for t in range(m.Nt) if len(set(T[t]) & set(T[t0])) == 1][0]
    for tp in (t0, shared, vert):
        I0, Ivv = dense.pair_integrals(m, [t0], [tp], k, n_out=16, n_in=6)
        # brute force: outer 12-point rule subdivided 4x, inner polar
        Vc, Vp = V[T[t0]], V[T[tp]]
        sub = []
        a, b, c = Vc
        ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
        for s1 in ([a, ab, ca], [ab, b, bc], [ca, bc, c], [ab, bc, ca]):
            s1 = np.array(s1)
            p, q, r_ = s1
            pq, qr, rp = (p + q) / 2, (q + r_) / 2, (r_ + p) / 2
            sub += [np.array(x) for x in ([p, pq, rp], [pq, q, qr], [rp, qr, r_], [pq, qr, rp])]
        bI0 = 0.0
        bIvv = np.zeros((3, 3), dtype=complex)
        for st in sub:
            X, w = map_rule(st, 8)
            for xq, wq in zip(X, w):
                f = lambda Y, R: np.concatenate(
                    [(np.exp(-1j * k * R) / (4 * np.pi * R))[:, None],
                     (Y - Vp[0]) * (np.exp(-1j * k * R) / (4 * np.pi * R))[:, None],
                     (Y - Vp[1]) * (np.exp(-1j * k * R) / (4 * np.pi * R))[:, None],
                     (Y - Vp[2]) * (np.exp(-1j * k * R) / (4 * np.pi * R))[:, None]], axis=1)
                inner = polar_integrate(xq, Vp, f, 24, 24, subdiv=3)
                bI0 += wq * inner[0]
                for i in range(3):
                    for j in range(3):
                        bIvv[i, j] += wq * np.dot(xq - Vc[i], inner[1 + 3 * j:4 + 3 * j])
        assert abs(I0[0] - bI0) / abs(bI0) < 1e-4, (tp, I0[0], bI0)
        assert np.abs(Ivv[0] - bIvv).max() / np.abs(bIvv).max() < 5e-4, tp


def test_default_close_rule_accuracy():
    """Default orders (n_out = n_in = 4) on coincident pairs stay within 1e-2 of
    a converged rule (the outer integrand has log-singular derivatives at the
    edges, so Gauss converges slowly; measured 3e-3 / 6e-3)."""
    import efie_inputs as E
    from oracle import dense
    from oracle.geometry import build_rwg
    V, T = E.icosphere(3, 0.5)
    m = build_rwg(V, T)
    c = np.arange(m.Nt)
    I0a, Iva = dense.pair_integrals(m, c, c, 2 * np.pi)
    I0b, Ivb = dense.pair_integrals(m, c, c, 2 * np.pi, n_out=12, n_in=8)
    assert np.abs(I0a - I0b).max() / np.abs(I0b).max() < 1e-2
    assert np.abs(Iva - Ivb).max() / np.abs(Ivb).max() < 1e-2
