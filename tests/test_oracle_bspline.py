"""Pins of the oracle's B-spline algebra (Sec. III-A, IV-B, V-B, Table I)
against identities that hold exactly: partition of unity, knot insertion
leaves the curve unchanged, transfer and stabilization matrices reproduce the
coarse splines, the p = 3 averaged-knot identity, Table I, and the growth of
||B^-1||_inf for equidistant vs stabilized knots."""
import os

import numpy as np
import pytest

from oracle import bspline as bs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_table1_golden():
    rows = [l.split() for l in open(os.path.join(GOLD, "table1_knots_to_remove.txt"))
            if l.strip() and not l.startswith("#")]
    assert {int(p): int(r) for p, r in rows} == bs.S_REMOVE


def test_eqknots_matches_definition():
    # Eq. eqknots on [0,1]: u_i = (i-p-1)/(s-p) for i in [p+2, s] (1-based)
    for p in range(1, 7):
        s = p + 5
        U = bs.open_knots(0.0, 1.0, s, p)
        ref = [0.0] * (p + 1) + [(i - p - 1) / (s - p) for i in range(p + 2, s + 1)] + [1.0] * (p + 1)
        assert np.allclose(U, ref, atol=0, rtol=0)


@pytest.mark.parametrize("p", range(1, 7))
def test_partition_of_unity(p):
    U = bs.open_knots(-1.0, 3.0, p + 6, p)
    x = np.linspace(-1, 3, 101)
    assert np.abs(bs.basis(U, p, x).sum(1) - 1).max() < 1e-14


@pytest.mark.parametrize("p", range(1, 7))
def test_knot_insertion_identity(p):
    rng = np.random.default_rng(p)
    U = bs.open_knots(0.0, 7.0, p + 7, p)
    w = rng.standard_normal(p + 7)
    x = rng.uniform(0, 7, 200)
    for ub in (0.5, 2.0, 3.3, 6.99):
        Ub, wb = bs.insert_knot(U, p, w, ub)
        assert np.abs(bs.basis(Ub, p, x) @ wb - bs.basis(U, p, x) @ w).max() < 1e-13


@pytest.mark.parametrize("p", range(1, 7))
@pytest.mark.parametrize("case", ["const", "increase"])
def test_transfer_matrix_exact(p, case):
    """Sec. IV-B: C[j,:] expresses parent spline j on each child's extended
    domain exactly (paper: errors ~1e-14, Sec. IV-E)."""
    s, sb = p + 4, 1
    sp = s + 2 * sb
    if case == "const":
        r, s_p, sb_p = 2, s, 1
    else:
        r, s_p, sb_p = 1, 2 * s - p, sb
    Up = bs.open_knots(-sb_p * r, (s_p - p + sb_p) * r, s_p + 2 * sb_p, p)
    rng = np.random.default_rng(10 * p)
    gold = float([l.split()[1] for l in open(os.path.join(GOLD, "paper_numbers.txt"))
                  if l.startswith("interlevel_transfer_max_rel_error")][0])
    for off in (0, s - p):
        Uc = bs.open_knots(off - sb, off + (s - p) + sb, sp, p)
        C = bs.restriction_matrix(Up, Uc, p)
        x = rng.uniform(Uc[0], Uc[-1], 300)
        err = np.abs(bs.basis(Uc, p, x) @ C.T - bs.basis(Up, p, x)).max()
        assert err < 10 * gold


@pytest.mark.parametrize("p", range(1, 7))
def test_stabilization_matrix_exact(p):
    sp = p + 6
    Ue = bs.open_knots(0.0, float(sp - p), sp, p)
    Us = bs.stabilized_knots(Ue, p, bs.S_REMOVE[p])
    assert len(Us) - p - 1 == sp - 2 * bs.S_REMOVE[p]
    S = bs.stabilization_matrix(Ue, Us, p)
    x = np.linspace(0, sp - p, 333)
    assert np.abs(bs.basis(Ue, p, x) @ S.T - bs.basis(Us, p, x)).max() < 1e-13
    # every stabilized knot is an equidistant knot (Sec. V-B)
    assert set(np.round(Us, 12)) <= set(np.round(Ue, 12))


def test_p3_stabilized_equals_averaged():
    """Sec. V-B: for p = 3 removing the knots i = p+2 and i = s gives the
    averaged knot vector (Eq. avgknots) with s_avg = s_eq - 2."""
    for s_eq in range(7, 25):
        Us = bs.stabilized_knots(bs.open_knots(0.0, 1.0, s_eq, 3), 3, 1)
        Ua = bs.averaged_knots(s_eq - 2, 3)
        assert np.abs(Us - Ua).max() < 1e-15


def test_sampling_inverse_norm_growth():
    """Fig. condition_number (qualitative): ||B^-1||_inf grows quickly with s for
    equidistant knots and stays bounded for stabilized ones."""
    for p in (3, 5):
        eq, st = [], []
        for s in (12, 20, 30):
            Ue = bs.open_knots(0.0, 1.0, s, p)
            Be = bs.sampling_matrix(Ue, p, bs.interpolation_points(0, 1, s))
            Us = bs.stabilized_knots(Ue, p, bs.S_REMOVE[p])
            ns = len(Us) - p - 1
            Bs = bs.sampling_matrix(Us, p, bs.interpolation_points(0, 1, ns))
            eq.append(np.abs(np.linalg.inv(Be)).sum(1).max())
            st.append(np.abs(np.linalg.inv(Bs)).sum(1).max())
        assert eq[2] > 4 * eq[0]
        assert st[2] < 1.5 * st[0]
        assert st[2] < eq[2] / 5


def test_projector_reproduces_polynomials():
    """P = B_stab^-1 S maps the equidistant moments of a degree-p polynomial's
    samples consistently: B_stab^T P^T-free check -- interpolating a spline in
    the stabilized space returns its own coefficients."""
    rng = np.random.default_rng(3)
    for p in range(1, 7):
        sp = p + 6
        Ue = bs.open_knots(0.0, float(sp - p), sp, p)
        P, S, B, x = bs.projector(Ue, p, bs.S_REMOVE[p])
        Us = bs.stabilized_knots(Ue, p, bs.S_REMOVE[p])
        c = rng.standard_normal(B.shape[0])
        vals = bs.basis(Us, p, x) @ c          # samples of a stabilized spline
        assert np.abs(np.linalg.solve(B.T, vals) - c).max() < 1e-10
        assert np.allclose(P, np.linalg.solve(B, S))
