"""Mie series for the surface current on a PEC sphere (oracle; test
infrastructure only).

Standard vector-spherical-harmonic solution (Bohren & Huffman 1983, Ch. 4,
perfect-conductor limit a_n = psi_n'(x)/xi_n'(x), b_n = psi_n(x)/xi_n(x)),
derived in the e^{-i w t} convention and conjugated to the paper's e^{j w t}
convention (Sec. II).  With the Riccati-Bessel Wronskian psi xi' - psi' xi = i
the total tangential field on r = a reduces to

    eta H_theta = (sin phi / x) sum_n E_n [ i pi_n / xi_n' - tau_n / xi_n ]
    eta H_phi   = (cos phi / x) sum_n E_n [ i tau_n / xi_n' - pi_n / xi_n ]

with E_n = i^n (2n+1)/(n(n+1)), x = ka, and the surface current (normalized
by the wave impedance, as j in Sec. II) is eta J = r_hat x eta H.
"""
from __future__ import annotations

import numpy as np
from scipy import special


def _riccati(nmax, x):
    n = np.arange(1, nmax + 1)
    jn = special.spherical_jn(n, x)
    jnp = special.spherical_jn(n, x, derivative=True)
    yn = special.spherical_yn(n, x)
    ynp = special.spherical_yn(n, x, derivative=True)
    psi = x * jn
    psip = jn + x * jnp
    xi = x * (jn + 1j * yn)
    xip = (jn + 1j * yn) + x * (jnp + 1j * ynp)
    return n, psi, psip, xi, xip


def _pi_tau(nmax, mu):
    """pi_n = P_n^1(cos t)/sin t and tau_n = d P_n^1/dt (B&H 4.47), n = 1..nmax."""
    P = mu.shape[0]
    pi = np.zeros((nmax + 1, P))
    tau = np.zeros((nmax + 1, P))
    pi[1] = 1.0
    tau[1] = mu
    for n in range(2, nmax + 1):
        pi[n] = ((2 * n - 1) / (n - 1)) * mu * pi[n - 1] - (n / (n - 1)) * pi[n - 2]
        tau[n] = n * mu * pi[n] - (n + 1) * pi[n - 1]
    return pi[1:], tau[1:]


def surface_current(points, radius, k, khat=(0.0, 0.0, 1.0), pol=(1.0, 0.0, 0.0), nmax=None):
    """eta*J (e^{j w t}) at points on the sphere |x| = radius centred at the
    origin, for the incident field e^i = pol * exp(-jk khat.x)."""
    points = np.asarray(points, dtype=np.float64)
    khat = np.asarray(khat, dtype=np.float64)
    khat = khat / np.linalg.norm(khat)
    pol = np.asarray(pol, dtype=np.float64)
    pol = pol - (pol @ khat) * khat
    pol = pol / np.linalg.norm(pol)
    ez, ex = khat, pol
    ey = np.cross(ez, ex)
    R = np.stack([ex, ey, ez])                     # rows: local axes
    loc = points @ R.T
    x = k * radius
    if nmax is None:
        nmax = int(np.ceil(x + 4.05 * x ** (1.0 / 3.0) + 10))
    n, psi, psip, xi, xip = _riccati(nmax, x)
    rr = np.linalg.norm(loc, axis=1)
    theta = np.arccos(np.clip(loc[:, 2] / rr, -1.0, 1.0))
    phi = np.arctan2(loc[:, 1], loc[:, 0])
    pi, tau = _pi_tau(nmax, np.cos(theta))
    En = (1j ** n) * (2 * n + 1) / (n * (n + 1))
    s1 = (En / xip)[:, None]
    s2 = (En / xi)[:, None]
    Ht = (np.sin(phi) / x) * np.sum(1j * pi * s1 - tau * s2, axis=0)
    Hp = (np.cos(phi) / x) * np.sum(1j * tau * s1 - pi * s2, axis=0)
    # e^{-iwt} -> e^{jwt}: conjugate phasors
    Jt = np.conj(-Hp)
    Jp = np.conj(Ht)
    st, ct, sp, cp = np.sin(theta), np.cos(theta), np.sin(phi), np.cos(phi)
    th_hat = np.stack([ct * cp, ct * sp, -st], axis=1)
    ph_hat = np.stack([-sp, cp, np.zeros_like(sp)], axis=1)
    J_loc = Jt[:, None] * th_hat + Jp[:, None] * ph_hat
    return J_loc @ R                               # back to global axes
