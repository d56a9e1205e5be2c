"""Pin of the Mie surface current (oracle/mie.py) that does not go through the
dense EFIE: the extinction theorem.  On a perfect conductor the induced
surface current J radiates the scattered field, and inside the sphere that
field cancels the incident one exactly:

    E_i(x) + E_s(x) = 0,   E_s(x) = -jk \\int (I + grad grad / k^2) g(x - x') eta J(x') dS'

for |x| < a, with g = exp(-jkR)/(4 pi R) and the e^{jwt} convention of the
incident field E_i = pol exp(-jk khat . x) (Sec. II).  A wrong sign, a
swapped angular function, a missing conjugation or a wrong series term in the
current leaves a non-zero interior field.  The surface integral runs on a
Gauss-Legendre (cos theta) x trapezoid (phi) rule, spectrally accurate for the
smooth integrand at interior points."""
import numpy as np
import pytest

from oracle import mie


def _sphere_rule(radius, n_theta, n_phi):
    mu, w = np.polynomial.legendre.leggauss(n_theta)
    phi = 2 * np.pi * np.arange(n_phi) / n_phi
    M, P = np.meshgrid(mu, phi, indexing="ij")
    st = np.sqrt(1 - M ** 2)
    pts = radius * np.stack([st * np.cos(P), st * np.sin(P), M], axis=-1).reshape(-1, 3)
    wts = (radius ** 2 * np.outer(w, np.full(n_phi, 2 * np.pi / n_phi))).reshape(-1)
    return pts, wts


def _radiated(x_obs, pts, wts, etaJ, k):
    """E_s at the observation points from the surface current etaJ."""
    out = np.zeros((len(x_obs), 3), dtype=np.complex128)
    for i, x in enumerate(x_obs):
        d = x[None, :] - pts
        R = np.linalg.norm(d, axis=1)
        rh = d / R[:, None]
        g = np.exp(-1j * k * R) / (4 * np.pi * R)
        kR = k * R
        a = 1 - (1 + 1j * kR) / kR ** 2
        b = (3 + 3j * kR - kR ** 2) / kR ** 2
        proj = np.sum(rh * etaJ, axis=1)
        field = (a[:, None] * etaJ + b[:, None] * proj[:, None] * rh) * (g * wts)[:, None]
        out[i] = -1j * k * field.sum(axis=0)
    return out


@pytest.mark.parametrize("ka, khat, pol", [
    (0.5, (0.0, 0.0, -1.0), (1.0, 0.0, 0.0)),
    (2.0, (0.3, -0.2, 0.9), (1.0, 0.4, 0.0)),
    (6.0, (-0.5, 0.7, 0.1), (0.2, 0.1, 1.0)),
])
def test_extinction_theorem(ka, khat, pol):
    radius = 1.0
    k = ka / radius
    n_theta = int(2 * ka) + 40
    pts, wts = _sphere_rule(radius, n_theta, 2 * n_theta)
    etaJ = mie.surface_current(pts, radius, k, khat, pol)
    khat_u = np.asarray(khat) / np.linalg.norm(khat)
    p = np.asarray(pol, dtype=float)
    p = p - (p @ khat_u) * khat_u
    p /= np.linalg.norm(p)
    # the current is tangential
    assert np.abs(np.sum(etaJ * pts, axis=1)).max() < 1e-12 * np.abs(etaJ).max()
    rng = np.random.default_rng(7)
    d = rng.standard_normal((8, 3))
    x_obs = d / np.linalg.norm(d, axis=1, keepdims=True) * rng.uniform(0.0, 0.5, (8, 1)) * radius
    Ei = p[None, :] * np.exp(-1j * k * (x_obs @ khat_u))[:, None]
    Es = _radiated(x_obs, pts, wts, etaJ, k)
    assert np.abs(Ei + Es).max() < 1e-10, np.abs(Ei + Es).max()   # measured 5e-15 - 2e-14
    # and the check has teeth: the current of the other time convention (no
    # conjugation), the current of the opposite sign and a series cut short
    # each leave an interior field (measured 1.6 - 2.6, 1.8 - 2.0, 4e-3 - 4e-2)
    for wrong in (np.conj(etaJ), -etaJ,
                  mie.surface_current(pts, radius, k, khat, pol, nmax=max(2, int(ka)))):
        assert np.abs(Ei + _radiated(x_obs, pts, wts, wrong, k)).max() > 1e-3


def test_low_frequency_limit():
    """As ka -> 0 the sphere sees a uniform incident magnetic field, whose
    tangential total field on a perfect conductor is 3/2 of the incident one:
    eta J -> (3/2) n x (khat x pol), with O(ka) corrections."""
    radius, khat, pol = 1.0, np.array([0.0, 0.6, 0.8]), np.array([1.0, 0.0, 0.0])
    pts, _ = _sphere_rule(radius, 12, 24)
    n = pts / radius
    J0 = 1.5 * np.cross(n, np.cross(khat, pol)[None, :])
    errs = []
    for ka in (1e-2, 1e-3):
        J = mie.surface_current(pts, radius, ka / radius, khat, pol)
        errs.append(np.abs(J - J0).max() / np.abs(J0).max())
    assert errs[1] < 3e-3 and errs[1] < 0.2 * errs[0]
