"""Spin Hamiltonians of eq. Ht (Sec. 2.2), built two independent ways.

Test infrastructure only (see ``oracle/__init__``).

* ``dense_hamiltonian``: sums Kronecker products of the complex 2x2 Pauli matrices,
  site 0 being the leftmost factor (Sec. 2.2, the sigma_i embedding), and returns
  the real part after checking the imaginary part vanishes.
* ``TensorHamiltonian``: applies the same operator without a matrix, by acting on
  the legs of the state viewed as an N-leg tensor (leg q = site q): X flips a leg,
  Z multiplies it by (+1, -1), and Y_a Y_b = -(X_a Z_a)(X_b Z_b) because Y = i X Z.
* ``hamiltonian_row``: one row of H from the Pauli action on a single basis vector
  (for sampled rows of Hamiltonians too large to build or apply whole).

Terms: for every pair a < b, Jx X_a X_b + Jy Y_a Y_b + Jz Z_a Z_b; for every site,
hz Z_q + gx X_q. A pair with one site in the system (sites < N_s) and one in the
bath is multiplied by lambda_sb (Sec. 5.5's epsilon).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

SX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
SY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
SZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)
PAULI = {"x": SX, "y": SY, "z": SZ}


def _is_sb(spec, a: int, b: int) -> bool:
    return (a < spec.n_sys) != (b < spec.n_sys)


def pair_terms(spec, part: str = "total"):
    """Yield (a, b, axis, coefficient) for the two-site terms of ``part``.

    ``part`` is "total", "sys" (both sites in the system), "bath" (both in the
    bath) or "sb" (one in each). lambda_sb is applied to system-bath pairs only.
    """
    n = spec.n_sites
    for a in range(n):
        for b in range(a + 1, n):
            sb = _is_sb(spec, a, b)
            in_sys = a < spec.n_sys and b < spec.n_sys
            kind = "sb" if sb else ("sys" if in_sys else "bath")
            if part != "total" and part != kind:
                continue
            scale = spec.lambda_sb if sb else 1.0
            for axis, table in (("x", spec.jx), ("y", spec.jy), ("z", spec.jz)):
                c = float(table[a, b]) * scale
                if c != 0.0:
                    yield a, b, axis, c


def site_terms(spec, part: str = "total"):
    """Yield (q, axis, coefficient) for the one-site field terms of ``part``."""
    for q in range(spec.n_sites):
        in_sys = q < spec.n_sys
        if part == "sb":
            return
        if part == "sys" and not in_sys:
            continue
        if part == "bath" and in_sys:
            continue
        for axis, vec in (("z", spec.hz), ("x", spec.gx)):
            c = float(vec[q])
            if c != 0.0:
                yield q, axis, c


def _embed(ops: dict, n: int):
    """Kronecker product over sites 0..n-1 (site 0 leftmost) of ops[q] or I."""
    out = sp.identity(1, dtype=np.complex128, format="csr")
    eye = sp.identity(2, dtype=np.complex128, format="csr")
    for q in range(n):
        m = sp.csr_matrix(ops[q]) if q in ops else eye
        out = sp.kron(out, m, format="csr")
    return out


def sparse_hamiltonian(spec, part: str = "total") -> sp.csr_matrix:
    """H (or one of its parts) as a real sparse matrix on all N sites."""
    n = spec.n_sites
    d = 1 << n
    acc = sp.csr_matrix((d, d), dtype=np.complex128)
    for a, b, axis, c in pair_terms(spec, part):
        acc = acc + c * _embed({a: PAULI[axis], b: PAULI[axis]}, n)
    for q, axis, c in site_terms(spec, part):
        acc = acc + c * _embed({q: PAULI[axis]}, n)
    acc = acc.tocsr()
    if acc.nnz:
        assert np.max(np.abs(acc.data.imag)) == 0.0, "Hamiltonian must be real"
    return sp.csr_matrix(acc.real)


def dense_hamiltonian(spec, part: str = "total") -> np.ndarray:
    return sparse_hamiltonian(spec, part).toarray()


def subsystem_hamiltonian(spec, which: str) -> np.ndarray:
    """Bare H_s (on the N_s system sites) or H_b (on the bath sites) alone."""
    n = spec.n_sites
    if which == "sys":
        sites = list(range(spec.n_sys))
    else:
        sites = list(range(spec.n_sys, n))
    m = len(sites)
    d = 1 << m
    acc = sp.csr_matrix((d, d), dtype=np.complex128)
    for a, b, axis, c in pair_terms(spec, which):
        acc = acc + c * _embed({sites.index(a): PAULI[axis], sites.index(b): PAULI[axis]}, m)
    for q, axis, c in site_terms(spec, which):
        acc = acc + c * _embed({sites.index(q): PAULI[axis]}, m)
    return np.asarray(acc.real.toarray())


def hamiltonian_row(spec, state: int, part: str = "total") -> dict:
    """Row ``state`` of H as {column: value}: the Pauli terms applied to one basis vector.

    H is real symmetric, so row s equals column s, H|s>. Site q is bit N-1-q of the
    state index (site 0 leftmost in the Kronecker order) and bit 0 is spin up:
    Z|b> = (-1)^b |b>, X|b> = |1-b>, Y|b> = i (-1)^b |1-b>, so a pair term
    X_a X_b flips both bits, Y_a Y_b flips both with the factor i^2 (-1)^(b_a + b_b),
    Z_a Z_b keeps the state with (-1)^(b_a + b_b). For rows of a Hamiltonian too large
    to build (sampled checks at full size).
    """
    n = spec.n_sites
    out: dict = {}

    def bit(q):
        return (state >> (n - 1 - q)) & 1

    def add(col, v):
        out[col] = out.get(col, 0.0) + v

    for a, b, axis, c in pair_terms(spec, part):
        flip = (1 << (n - 1 - a)) | (1 << (n - 1 - b))
        sgn = -1.0 if (bit(a) + bit(b)) % 2 else 1.0
        if axis == "x":
            add(state ^ flip, c)
        elif axis == "y":
            add(state ^ flip, -c * sgn)
        else:
            add(state, c * sgn)
    for q, axis, c in site_terms(spec, part):
        if axis == "z":
            add(state, -c if bit(q) else c)
        else:
            add(state ^ (1 << (n - 1 - q)), c)
    return out


class TensorHamiltonian:
    """Matrix-free H x for x of shape (2^N, B), acting on tensor legs."""

    def __init__(self, spec, part: str = "total"):
        self.spec = spec
        self.n = spec.n_sites
        self.part = part
        self.pairs = list(pair_terms(spec, part))
        self.sites = list(site_terms(spec, part))
        self._diag = None

    def _sign(self, q: int) -> np.ndarray:
        shape = [1] * (self.n + 1)
        shape[q] = 2
        return np.array([1.0, -1.0]).reshape(shape)

    def diagonal(self) -> np.ndarray:
        """The Z-only part of H as a vector of length 2^N."""
        if self._diag is None:
            shape = (2,) * self.n + (1,)
            dg = np.zeros(shape)
            for a, b, axis, c in self.pairs:
                if axis == "z":
                    dg = dg + c * (self._sign(a) * self._sign(b))
            for q, axis, c in self.sites:
                if axis == "z":
                    dg = dg + c * self._sign(q)
            self._diag = np.broadcast_to(dg, shape).reshape(-1).copy()
        return self._diag

    def __call__(self, x: np.ndarray) -> np.ndarray:
        x = np.asarray(x, dtype=np.float64)
        squeeze = x.ndim == 1
        if squeeze:
            x = x[:, None]
        bcols = x.shape[1]
        t = x.reshape((2,) * self.n + (bcols,))
        y = self.diagonal()[:, None] * x
        yt = y.reshape(t.shape)
        for a, b, axis, c in self.pairs:
            if axis == "x":
                yt += c * np.flip(np.flip(t, a), b)
            elif axis == "y":
                # Y_a Y_b = (i X_a Z_a)(i X_b Z_b) = -(X_a Z_a)(X_b Z_b)
                zz = t * (self._sign(a) * self._sign(b))
                yt -= c * np.flip(np.flip(zz, a), b)
        for q, axis, c in self.sites:
            if axis == "x":
                yt += c * np.flip(t, q)
        return y[:, 0] if squeeze else y

    def norm_bound(self) -> float:
        """sum of |coefficients|: an upper bound on ||H||_2 (each Pauli string has norm 1)."""
        return float(sum(abs(c) for *_, c in self.pairs) + sum(abs(c) for *_, c in self.sites))
