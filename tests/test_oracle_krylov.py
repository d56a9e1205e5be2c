"""Pins of the oracle's restarted flexible GMRES (`oracle.krylov.fgmres`), the
solver the learned preconditioner runs in, on seeded complex systems whose
solutions a library routine gives directly (LU):
  * with the exact inverse as preconditioner it converges in one iteration
    (the Krylov space of T M = I is spanned by b);
  * a fixed right preconditioner M gives the solution of T x = b (not of
    T M y = b): x = M y is returned;
  * a preconditioner that changes from one iteration to the next (flexible)
    still converges to that solution, with the true residual as reported;
  * restarts: a restart length far below the iteration count still converges;
  * a zero right-hand side returns x = 0 without iterating."""
import numpy as np

from oracle import krylov


def _system(n, seed):
    r = np.random.default_rng(seed)
    # well-conditioned complex non-Hermitian matrix: identity plus a scaled random part
    T = np.eye(n) + 0.3 * (r.standard_normal((n, n)) + 1j * r.standard_normal((n, n))) / np.sqrt(n)
    b = r.standard_normal(n) + 1j * r.standard_normal(n)
    return T, b


def _res(T, x, b):
    return np.linalg.norm(b - T @ x) / np.linalg.norm(b)


def test_exact_inverse_one_iteration():
    T, b = _system(60, 1)
    Ti = np.linalg.inv(T)
    x, info = krylov.fgmres(lambda v: T @ v, b, tol=1e-10, restart=20, precond=lambda v: Ti @ v)
    assert info["converged"] and info["iterations"] == 1
    assert np.linalg.norm(x - np.linalg.solve(T, b)) / np.linalg.norm(x) < 1e-12


def test_fixed_right_preconditioner():
    T, b = _system(80, 2)
    d = 1.0 / np.diag(T)
    x, info = krylov.fgmres(lambda v: T @ v, b, tol=1e-10, restart=40, precond=lambda v: d * v)
    xs = np.linalg.solve(T, b)
    assert info["converged"] and abs(info["true_rel_residual"] - _res(T, x, b)) < 1e-14
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-8


def test_flexible_preconditioner():
    T, b = _system(80, 3)
    calls = [0]

    def precond(v):
        # a different diagonal scaling at every call
        calls[0] += 1
        s = 1.0 + 0.5 * np.sin(np.arange(v.shape[0]) + calls[0])
        return s * v

    x, info = krylov.fgmres(lambda v: T @ v, b, tol=1e-10, restart=40, precond=precond)
    assert info["converged"] and calls[0] == info["iterations"]
    assert np.linalg.norm(x - np.linalg.solve(T, b)) / np.linalg.norm(x) < 1e-8
    assert abs(info["true_rel_residual"] - _res(T, x, b)) < 1e-14


def test_short_restarts():
    T, b = _system(100, 4)
    x, info = krylov.fgmres(lambda v: T @ v, b, tol=1e-10, restart=5, max_iters=2000)
    assert info["converged"] and info["iterations"] > 5 and _res(T, x, b) <= 1e-10


def test_zero_rhs():
    T, _ = _system(20, 5)
    x, info = krylov.fgmres(lambda v: T @ v, np.zeros(20, dtype=np.complex128))
    assert info["converged"] and info["iterations"] == 0 and not x.any()
