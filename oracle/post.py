"""Post-processing of rho*: H* and the von Neumann entropy.

Test infrastructure only (see ``oracle/__init__``).

* ``mean_force``: -(1/beta) ln(rho*) through the eigendecomposition of rho*
  (Sec. 3.2: transform eigenvalues instead of taking a matrix logarithm). With
  ``ln_z_star`` given it returns the absolute H* = -(1/beta) ln(Z* rho*) (eq. 6-7);
  without it, H* up to the additive constant -(1/beta) ln Z*.
* ``entropy``: S = -tr(rho ln rho) = -sum p ln p with 0 ln 0 = 0 (Sec. 5.3.1).
* ``energy_deviation``: tr(H* rho*) - tr(H_s rho_s), rho_s the Gibbs state of the bare
  system Hamiltonian H_s (Sec. 5.3.2, eq. deviation_of_Hamiltonian).
"""
from __future__ import annotations

import numpy as np


def mean_force(rho: np.ndarray, beta: float, ln_z_star: float | None = None) -> np.ndarray:
    w, u = np.linalg.eigh(0.5 * (rho + rho.T))
    if np.any(w <= 0):
        raise ValueError("rho* is not positive definite; ln is undefined")
    lw = np.log(w)
    if ln_z_star is not None:
        lw = lw + ln_z_star
    return -(u * lw) @ u.T / beta


def entropy(rho: np.ndarray) -> float:
    w = np.linalg.eigvalsh(0.5 * (rho + rho.T))
    w = w[w > 0]
    return float(-np.sum(w * np.log(w)))


def energy_deviation(rho_star: np.ndarray, h_star: np.ndarray, h_s: np.ndarray, beta: float) -> float:
    w, u = np.linalg.eigh(0.5 * (h_s + h_s.T))
    f = np.exp(-beta * (w - w[0]))
    rho_s = (u * (f / f.sum())) @ u.T
    return float(np.trace(h_star @ rho_star) - np.trace(h_s @ rho_s))
