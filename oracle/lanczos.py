"""O2/O3: the paper's estimator, same seeds, written as plain float64 NumPy.

Test infrastructure only (see ``oracle/__init__``).

Algorithm 1 (block Lanczos), for j = 1..k with Q_0 = 0, B_0 = 0, Q_1 = V:
    Z   = H Q_j - Q_{j-1} B_{j-1}^T
    A_j = Q_j^T Z
    Z   = Z - Q_j A_j
    (Q_{j+1}, B_j) = qr(Z)
builds the block tridiagonal T (A_j on the diagonal, B_j below, B_j^T above).

From T (eq. fT, trB_est, rho_est and the E0 shift of Sec. 3.2):
    quadrature form  G_l = E1^T exp(-beta (T_l - E0)) E1
    Gram form        psi_l = Q_l exp(-beta (T_l - E0)/2) E1,  G_l = psi_l^T psi_l
    rho* ~ sum_l G_l / tr(sum_l G_l)
    ln Z_t ~ ln(d_b tr(sum_l G_l) / n_v) - beta E0
The Gram form is the function-application (Lanczos-FA) reading of the sqrt(rho)
construction of Sec. 2.1; it equals the quadrature form when Q^T Q = I.

Readings where the paper is silent (used identically by the CUDA library):
  * A_j is symmetrised, (A_j + A_j^T)/2 (exact arithmetic makes it symmetric);
  * qr(Z) is the thin QR with non-negative diagonal, computed column by column
    (classical Gram-Schmidt applied twice); a column whose remaining norm r
    satisfies r <= max(tau_abs * ||H||_bound, tau_rel * ||z_c||) is dropped
    (its Q column and its row of R set to zero) -- Krylov breakdown/deflation;
  * E0 = the smallest eigenvalue of all T_l (common to all l);
  * each bath vector runs its own recurrence of block size d_s (eq. trB_est);
    ``run(..., block=False)`` instead runs one recurrence of block size 1 per
    column e_i (x) v_l (the per-vector variant of Sec. 4.2).
"""
from __future__ import annotations

import numpy as np

from .rng import bath_vector, starting_block
from .spin_ops import TensorHamiltonian

TAU_ABS = 1e-12
TAU_REL = 1e-7


def qr_drop(z: np.ndarray, abs_tol: float, rel_tol: float):
    """Thin QR with non-negative diagonal; numerically dependent columns dropped."""
    d, p = z.shape
    q = np.zeros((d, p))
    r = np.zeros((p, p))
    kept = []
    for c in range(p):
        w = z[:, c].copy()
        nz = float(np.sqrt(w @ w))
        for _ in range(2):
            if kept:
                qk = q[:, kept]
                coef = qk.T @ w
                w = w - qk @ coef
                r[kept, c] += coef
        nr = float(np.sqrt(w @ w))
        if nr <= max(abs_tol, rel_tol * nz):
            continue  # dropped: q_c = 0, R[c, c] = 0, and row c of R stays zero
        q[:, c] = w / nr
        r[c, c] = nr
        kept.append(c)
    return q, r


def block_lanczos(apply_h, v: np.ndarray, k: int, hnorm: float,
                  tau_abs: float = TAU_ABS, tau_rel: float = TAU_REL):
    """Algorithm 1. Yields (j, Q_j, A_j, B_j) for j = 1..k (B_j couples Q_{j+1})."""
    d, p = v.shape
    q_prev = np.zeros((d, p))
    b_prev = np.zeros((p, p))
    q = v.copy()
    for j in range(1, k + 1):
        z = apply_h(q) - q_prev @ b_prev.T
        a = q.T @ z
        a = 0.5 * (a + a.T)
        z = z - q @ a
        q_next, b = qr_drop(z, tau_abs * hnorm, tau_rel)
        yield j, q, a, b
        q_prev, q, b_prev = q, q_next, b


def assemble_t(a_blocks, b_blocks) -> np.ndarray:
    """Block tridiagonal T (k*p square) from A_1..A_k and B_1..B_{k-1}."""
    k = len(a_blocks)
    p = a_blocks[0].shape[0]
    t = np.zeros((k * p, k * p))
    for j in range(k):
        t[j * p:(j + 1) * p, j * p:(j + 1) * p] = a_blocks[j]
        if j + 1 < k:
            t[(j + 1) * p:(j + 2) * p, j * p:(j + 1) * p] = b_blocks[j]
            t[j * p:(j + 1) * p, (j + 1) * p:(j + 2) * p] = b_blocks[j].T
    return t


def lanczos_coefficients(apply_h, v, k, hnorm):
    """(A_1..A_k, B_1..B_k) of Algorithm 1 for starting block v."""
    a_list, b_list = [], []
    for _, _, a, b in block_lanczos(apply_h, v, k, hnorm):
        a_list.append(a)
        b_list.append(b)
    return a_list, b_list


def function_of_t_first_block(t: np.ndarray, p: int, func):
    """func(T) E1 (k*p x p) through the eigendecomposition of T."""
    w, u = np.linalg.eigh(t)
    return (u * func(w)) @ u[:p, :].T


def psi_gram_form(apply_h, v, k, hnorm, coef_blocks):
    """sum_j Q_j C_j for each C in ``coef_blocks`` (list of (k*p, p) arrays).

    Re-runs Algorithm 1 (deterministic, identical Q_j) so no basis is stored.
    """
    p = v.shape[1]
    psis = [np.zeros_like(v) for _ in coef_blocks]
    for j, q, _, _ in block_lanczos(apply_h, v, k, hnorm):
        for psi, c in zip(psis, coef_blocks):
            psi += q @ c[(j - 1) * p:j * p, :]
    return psis


class Estimator:
    """The paper's estimator for one model, same seeds as the library."""

    def __init__(self, spec, apply_h=None, hnorm=None):
        self.spec = spec
        ham = TensorHamiltonian(spec)
        self.apply_h = apply_h if apply_h is not None else ham
        self.hnorm = hnorm if hnorm is not None else ham.norm_bound()

    def starting_block(self, l: int, seed: int, dist: str) -> np.ndarray:
        s = self.spec
        return starting_block(s.d_s, bath_vector(s.d_b, l, seed, dist))

    def run(self, betas, n_v: int, k: int, seed: int, dist: str, vectors=None,
            gram: bool = True, e0=None, block: bool = True):
        """Returns a dict with rho, lnZ (Gram form), rho_quad, per-l grams, E0, T.

        ``vectors`` restricts the run to a subset of bath-vector indices (the
        estimator is a sum over l, so any subset can be checked on its own);
        ``e0`` then supplies the shift the full run used. ``block=False`` runs the
        regular (block size 1) Lanczos algorithm on each column of the starting
        block separately (Sec. 4.2, the alternative to block Lanczos).
        """
        if not block:
            return self._run_single(betas, n_v, k, seed, dist)
        s = self.spec
        p = s.d_s
        betas = np.atleast_1d(np.asarray(betas, dtype=np.float64))
        ls = list(range(n_v)) if vectors is None else list(vectors)
        t_list, v_list = {}, {}
        for l in ls:
            v = self.starting_block(l, seed, dist)
            a, b = lanczos_coefficients(self.apply_h, v, k, self.hnorm)
            t_list[l] = (a, b)
            v_list[l] = v
        ts = {l: assemble_t(*t_list[l]) for l in ls}
        if e0 is None:
            e0 = min(float(np.linalg.eigvalsh(ts[l])[0]) for l in ls)
        quad = np.zeros((len(betas), len(ls), p, p))
        grams = np.zeros((len(betas), len(ls), p, p))
        for li, l in enumerate(ls):
            coefs = []
            for bi, beta in enumerate(betas):
                c = function_of_t_first_block(ts[l], p, lambda x: np.exp(-beta * (x - e0) / 2.0))
                quad[bi, li] = c.T @ c
                coefs.append(c)
            if gram:
                psis = psi_gram_form(self.apply_h, v_list[l], k, self.hnorm, coefs)
                for bi, psi in enumerate(psis):
                    grams[bi, li] = psi.T @ psi
        out = dict(e0=e0, quad_l=quad, betas=betas, T={l: t_list[l] for l in ls})
        out["rho_quad"], out["lnZ_quad"] = _normalise(quad, betas, e0, s.d_b, len(ls))
        if gram:
            out["gram_l"] = grams
            out["rho"], out["lnZ"] = _normalise(grams, betas, e0, s.d_b, len(ls))
        return out


    def _run_single(self, betas, n_v: int, k: int, seed: int, dist: str):
        """Per-column Lanczos: for starting column v_i = e_i (x) v_l, T_{l,i} from
        Algorithm 1 with block size 1; psi_{l,i} = Q_{l,i} exp(-beta (T_{l,i} - E0)/2) e1
        and G_l[i, j] = psi_{l,i}^T psi_{l,j} (Gram form). The quadrature form has only
        the diagonal e1^T exp(-beta (T_{l,i} - E0)) e1 (its off-diagonal entries are
        not estimated by single-vector quadrature and are left zero). E0 is the
        smallest eigenvalue of all T_{l,i}."""
        s = self.spec
        p = s.d_s
        betas = np.atleast_1d(np.asarray(betas, dtype=np.float64))
        cols, ts = {}, {}
        for l in range(n_v):
            v = self.starting_block(l, seed, dist)
            for i in range(p):
                cols[l, i] = v[:, i:i + 1]
                ts[l, i] = assemble_t(*lanczos_coefficients(self.apply_h, cols[l, i], k, self.hnorm))
        e0 = min(float(np.linalg.eigvalsh(t)[0]) for t in ts.values())
        quad = np.zeros((len(betas), n_v, p, p))
        grams = np.zeros((len(betas), n_v, p, p))
        for l in range(n_v):
            psis = []
            for i in range(p):
                coefs = []
                for bi, beta in enumerate(betas):
                    c = function_of_t_first_block(ts[l, i], 1, lambda x: np.exp(-beta * (x - e0) / 2.0))
                    quad[bi, l, i, i] = float((c.T @ c)[0, 0])
                    coefs.append(c)
                psis.append(psi_gram_form(self.apply_h, cols[l, i], k, self.hnorm, coefs))
            for bi in range(len(betas)):
                m = np.hstack([psis[i][bi] for i in range(p)])
                grams[bi, l] = m.T @ m
        out = dict(e0=e0, quad_l=quad, gram_l=grams, betas=betas)
        out["rho_quad"], out["lnZ_quad"] = _normalise(quad, betas, e0, s.d_b, n_v)
        out["rho"], out["lnZ"] = _normalise(grams, betas, e0, s.d_b, n_v)
        return out


def _normalise(g_l, betas, e0, d_b, n_v):
    tot = g_l.sum(axis=1)
    tr = np.trace(tot, axis1=1, axis2=2)
    rho = tot / tr[:, None, None]
    lnz = np.log(d_b * tr / n_v) - betas * e0
    return rho, lnz


def exact_function_estimator(spec, h_dense, betas, n_v, seed, dist):
    """O2: eq. rho_est's first line (exact exp(-beta H/2), same bath vectors)."""
    w, u = np.linalg.eigh(h_dense)
    e = float(w[0])
    betas = np.atleast_1d(betas)
    rhos, lnz = [], []
    for beta in betas:
        half = (u * np.exp(-beta * (w - e) / 2.0)) @ u.T
        g = np.zeros((spec.d_s, spec.d_s))
        for l in range(n_v):
            psi = half @ starting_block(spec.d_s, bath_vector(spec.d_b, l, seed, dist))
            g += psi.T @ psi
        tr = np.trace(g)
        rhos.append(g / tr)
        lnz.append(np.log(spec.d_b * tr / n_v) - beta * e)
    return np.array(rhos), np.array(lnz)
