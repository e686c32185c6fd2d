"""App. C: closed-form rho* eigenvalues for the isotropic XY chain, N_s = 2.

Test infrastructure only (see ``oracle/__init__``).

Model (checked against exact diagonalisation in the tests): the open chain
H = (J/2) sum_{i=1}^{N-1} (X_i X_{i+1} + Y_i Y_{i+1}) + (h/2) sum_i Z_i.

Readings of garbled formulas in App. C:
  * N_k = 1 / (1 + exp(beta lambda_k)) (a parenthesis is misplaced in the text);
  * <sigma_j^z> = 1 - (4/(N+1)) sum_k sin^2(j k pi/(N+1)) N_k (the leading "1 -"
    is missing in the text); the overall sign of <sigma^z> only swaps p_1 and p_4,
    so the eigenvalue *set* does not depend on it;
  * delta uses <sigma_1^z> (an opening bracket is missing).
"""
from __future__ import annotations

import numpy as np


def _lam(n: int, j: float, h: float) -> np.ndarray:
    k = np.arange(1, n + 1)
    return h - 2.0 * j * np.cos(k * np.pi / (n + 1))


def rho_eigenvalues(n: int, beta: float, j: float = 1.0, h: float = 0.3) -> np.ndarray:
    """p_1..p_4 of App. C, sorted ascending."""
    k = np.arange(1, n + 1)
    lam = _lam(n, j, h)
    occ = 1.0 / (1.0 + np.exp(beta * lam))
    th = k * np.pi / (n + 1)
    sxx = -4.0 / (n + 1) * np.sum(np.sin(th) * np.sin(2 * th) * occ)
    sz1 = 1.0 - 4.0 / (n + 1) * np.sum(np.sin(1 * th) ** 2 * occ)
    sz2 = 1.0 - 4.0 / (n + 1) * np.sum(np.sin(2 * th) ** 2 * occ)
    szz = sz1 * sz2 - sxx ** 2
    delta = np.sqrt(4.0 * sxx ** 2 + (sz1 - sz2) ** 2)
    p = np.array([
        (1 + sz1 + sz2 + szz) / 4,
        (1 - delta - szz) / 4,
        (1 + delta - szz) / 4,
        (1 - sz1 - sz2 + szz) / 4,
    ])
    return np.sort(p)


def log_partition_chain(n: int, beta: float, j: float = 1.0, h: float = 0.3) -> float:
    """ln Z_N = beta N h / 2 + sum_k ln(1 + exp(-beta lambda_k))."""
    lam = _lam(n, j, h)
    return float(beta * n * h / 2.0 + np.sum(np.logaddexp(0.0, -beta * lam)))


def mean_energy_chain(n: int, beta: float, j: float = 1.0, h: float = 0.3) -> float:
    """<H> = -d ln Z_N / d beta = -N h / 2 + sum_k lambda_k / (1 + exp(beta lambda_k))."""
    lam = _lam(n, j, h)
    return float(-n * h / 2.0 + np.sum(lam / (1.0 + np.exp(beta * lam))))


def log_z_star(n: int, beta: float, j: float = 1.0, h: float = 0.3) -> float:
    """ln Z* = ln Z_N - ln Z_{N-2} (system = first two sites, bath = the open chain rest)."""
    return log_partition_chain(n, beta, j, h) - log_partition_chain(n - 2, beta, j, h)


def mean_force_eigenvalues(n: int, beta: float, j: float = 1.0, h: float = 0.3) -> np.ndarray:
    """h_j = -(1/beta) ln(Z* p_j), sorted to match ascending p (descending h)."""
    p = rho_eigenvalues(n, beta, j, h)
    return -(log_z_star(n, beta, j, h) + np.log(p)) / beta
