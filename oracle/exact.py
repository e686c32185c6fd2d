"""O1: the naive method (Sec. 2.4) -- exact diagonalisation plus an explicit partial trace.

Test infrastructure only (see ``oracle/__init__``).

rho*(beta) = tr_b(exp(-beta H_t)) / Z_t (eq. 4 with eq. 2-3), the partial trace
written out as the sum over bath basis states of (I_s x <b|) A (I_s x |b>) (Sec. 2.1).
The exponential is formed from the eigendecomposition with the smallest eigenvalue
subtracted, so ln Z_t = ln tr R - beta * lambda_min.
"""
from __future__ import annotations

import numpy as np

from .spin_ops import dense_hamiltonian, subsystem_hamiltonian


def partial_trace_bath(m: np.ndarray, d_s: int, d_b: int) -> np.ndarray:
    """R[i, j] = sum_b M[i*d_b + b, j*d_b + b] (system = leading tensor factor)."""
    r = np.zeros((d_s, d_s), dtype=m.dtype)
    for i in range(d_s):
        for j in range(d_s):
            r[i, j] = sum(m[i * d_b + b, j * d_b + b] for b in range(d_b)) if d_b <= 64 else \
                np.trace(m[i * d_b:(i + 1) * d_b, j * d_b:(j + 1) * d_b])
    return r


class ExactSolver:
    """Diagonalises H_t once and answers rho*, ln Z_t for any beta."""

    def __init__(self, spec):
        self.spec = spec
        self.h = dense_hamiltonian(spec)
        self.evals, self.evecs = np.linalg.eigh(self.h)
        self.lmin = float(self.evals[0])

    def exp_shifted(self, beta: float, power: float = 1.0) -> np.ndarray:
        """U exp(-power*beta*(Lambda - lambda_min)) U^T."""
        w = np.exp(-power * beta * (self.evals - self.lmin))
        return (self.evecs * w) @ self.evecs.T

    def reduced(self, beta: float):
        """(rho*, ln Z_t) at inverse temperature beta."""
        s = self.spec
        r = partial_trace_bath(self.exp_shifted(beta), s.d_s, s.d_b)
        tr = float(np.trace(r))
        return r / tr, float(np.log(tr) - beta * self.lmin)

    def ground_state_reduced(self, degeneracy_tol: float = 1e-9) -> np.ndarray:
        """beta -> infinity limit (Sec. 2.3): average of tr_b|psi_i><psi_i| over ground states."""
        s = self.spec
        idx = np.nonzero(self.evals <= self.lmin + degeneracy_tol)[0]
        acc = np.zeros((s.d_s, s.d_s))
        for i in idx:
            m = self.evecs[:, i].reshape(s.d_s, s.d_b)
            acc += m @ m.T
        return acc / len(idx)


def exact_rho(spec, betas):
    """rho*(beta) for each beta, shape (n_beta, d_s, d_s), and ln Z_t, shape (n_beta,)."""
    solver = ExactSolver(spec)
    rhos, lnz = [], []
    for b in np.atleast_1d(betas):
        r, z = solver.reduced(float(b))
        rhos.append(r)
        lnz.append(z)
    return np.array(rhos), np.array(lnz)


def bare_system_gibbs(spec, beta: float) -> np.ndarray:
    """exp(-beta H_s)/Z_s on the system alone (the H_sb = 0 answer, eq. HMF)."""
    hs = subsystem_hamiltonian(spec, "sys")
    w, u = np.linalg.eigh(hs)
    e = (u * np.exp(-beta * (w - w[0]))) @ u.T
    return e / np.trace(e)


def bath_log_partition(spec, beta: float) -> float:
    """ln Z_b = ln tr exp(-beta H_b) by exact diagonalisation of the bare bath."""
    hb = subsystem_hamiltonian(spec, "bath")
    w = np.linalg.eigvalsh(hb)
    return float(np.log(np.sum(np.exp(-beta * (w - w[0])))) - beta * w[0])
