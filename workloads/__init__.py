"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the estimator. It only writes down the spin
models the paper studies (eq. Ht, Sec. 2.2; the epsilon-scaled coupling of Sec. 5.5)
as plain coupling tables, plus temperature grids and the request stream used for
the serving workload. Both sides (the CPU oracle and the CUDA library) consume the
same ``ModelSpec`` and build their own operator from it.

Conventions (readings of Sec. 2.2, eq. Ht):
  * sigma are Pauli matrices (eigenvalues +-1); a coupling J[i, j] is stated once
    per unordered pair i < j (entries with i >= j are ignored);
  * sites are numbered 0..N-1, site 0 is the leftmost Kronecker factor, the system
    is sites 0..N_s-1 and the bath is the rest;
  * ``hz[q]`` is the coefficient of Z_q (the paper's h/2), ``gx[q]`` that of X_q;
  * ``lambda_sb`` multiplies every term that couples a system site with a bath
    site (the paper's epsilon of Sec. 5.5).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "ModelSpec",
    "xxz_chain",
    "xy_open_chain",
    "long_range_xxz",
    "long_range_tfim",
    "random_model",
    "spin_ladder",
    "bath_spec",
    "beta_grid",
    "config_c1",
    "config_c2",
    "config_c3",
    "config_c5",
    "serving_requests",
]


@dataclasses.dataclass
class ModelSpec:
    """A real spin-1/2 Hamiltonian given by its couplings (eq. Ht)."""

    n_sites: int
    n_sys: int
    jx: np.ndarray  # (N, N) float64, upper triangle used
    jy: np.ndarray
    jz: np.ndarray
    hz: np.ndarray  # (N,)
    gx: np.ndarray  # (N,)
    lambda_sb: float = 1.0
    name: str = ""

    @property
    def dim(self) -> int:
        return 1 << self.n_sites

    @property
    def d_s(self) -> int:
        return 1 << self.n_sys

    @property
    def d_b(self) -> int:
        return 1 << (self.n_sites - self.n_sys)

    def with_lambda(self, lam: float) -> "ModelSpec":
        return dataclasses.replace(self, lambda_sb=float(lam))


def _empty(n: int):
    z = np.zeros((n, n), dtype=np.float64)
    return z.copy(), z.copy(), z.copy(), np.zeros(n), np.zeros(n)


def xxz_chain(n: int, n_sys: int, j: float = 1.0, delta: float = 0.5, h: float = 0.0,
              lam: float = 1.0, periodic: bool = True) -> ModelSpec:
    """Nearest-neighbour XXZ chain J (XX + YY + Delta ZZ) + (h/2) sum Z."""
    jx, jy, jz, hz, gx = _empty(n)
    bonds = [(q, q + 1) for q in range(n - 1)]
    if periodic and n > 2:
        bonds.append((0, n - 1))
    for a, b in bonds:
        jx[a, b] += j
        jy[a, b] += j
        jz[a, b] += j * delta
    hz[:] = h / 2.0
    return ModelSpec(n, n_sys, jx, jy, jz, hz, gx, lam, f"xxz_chain_N{n}")


def xy_open_chain(n: int, n_sys: int, j: float = 1.0, h: float = 0.3) -> ModelSpec:
    """Open isotropic XY chain with coefficient J/2 on XX + YY and (h/2) on Z.

    This is the convention under which the closed form of App. C holds.
    """
    jx, jy, jz, hz, gx = _empty(n)
    for q in range(n - 1):
        jx[q, q + 1] = j / 2.0
        jy[q, q + 1] = j / 2.0
    hz[:] = h / 2.0
    return ModelSpec(n, n_sys, jx, jy, jz, hz, gx, 1.0, f"xy_open_N{n}")


def long_range_xxz(n: int, n_sys: int, alpha: float, delta: float = 1.0, h: float = 0.0,
                   lam: float = 1.0, j: float = 1.0) -> ModelSpec:
    """J_ij = J/|i-j|^alpha on XX + YY + Delta ZZ for all pairs (open chain)."""
    jx, jy, jz, hz, gx = _empty(n)
    for a in range(n):
        for b in range(a + 1, n):
            c = j / float(b - a) ** alpha
            jx[a, b] = c
            jy[a, b] = c
            jz[a, b] = c * delta
    hz[:] = h / 2.0
    return ModelSpec(n, n_sys, jx, jy, jz, hz, gx, lam, f"lr_xxz_N{n}_a{alpha}")


def long_range_tfim(n: int, n_sys: int, alpha: float, g: float, lam: float = 1.0,
                    j: float = 1.0) -> ModelSpec:
    """sum_{i<j} J/|i-j|^alpha Z_i Z_j + g sum X_i."""
    jx, jy, jz, hz, gx = _empty(n)
    for a in range(n):
        for b in range(a + 1, n):
            jz[a, b] = j / float(b - a) ** alpha
    gx[:] = g
    return ModelSpec(n, n_sys, jx, jy, jz, hz, gx, lam, f"lr_tfim_N{n}_g{g:.3f}")


def bath_spec(spec: ModelSpec) -> ModelSpec:
    """The bare bath of ``spec`` (its bath sites and the couplings among them) as a
    model with no system sites; bath site q of ``spec`` becomes site q - n_sys."""
    s = spec.n_sys
    return ModelSpec(spec.n_sites - s, 0, spec.jx[s:, s:].copy(), spec.jy[s:, s:].copy(),
                     spec.jz[s:, s:].copy(), spec.hz[s:].copy(), spec.gx[s:].copy(), 1.0,
                     (spec.name + "_bath") if spec.name else "bath")


def spin_ladder(n_rungs: int, system_rung: int, j_leg: float = 1.0, j_rung: float = -0.45,
                h: float = 1.0, lam: float = 1.0, numbering: str = "rung") -> ModelSpec:
    """Isotropic XY spin ladder of Sec. 5.2: two legs of n_rungs spins, coupling j_leg
    along the legs and j_rung on the rungs (J^x = J^y, J^z = 0), field (h/2) sum Z.
    The system is the rung `system_rung` (its two spins are sites 0 and 1); the bath
    sites follow rung by rung, leg 0 before leg 1 on each rung (numbering="rung"), or
    all of leg 0, then all of leg 1 (numbering="leg")."""
    n = 2 * n_rungs
    order = [(0, system_rung), (1, system_rung)]
    if numbering == "rung":
        order += [(leg, r) for r in range(n_rungs) if r != system_rung for leg in (0, 1)]
    else:
        order += [(leg, r) for leg in (0, 1) for r in range(n_rungs) if r != system_rung]
    site = {ls: q for q, ls in enumerate(order)}
    jx, jy, jz, hz, gx = _empty(n)

    def bond(a, b, c):
        i, k = sorted((site[a], site[b]))
        jx[i, k] += c
        jy[i, k] += c
    for r in range(n_rungs):
        bond((0, r), (1, r), j_rung)
        if r + 1 < n_rungs:
            bond((0, r), (0, r + 1), j_leg)
            bond((1, r), (1, r + 1), j_leg)
    hz[:] = h / 2.0
    return ModelSpec(n, 2, jx, jy, jz, hz, gx, lam, f"ladder_L{n_rungs}_sys{system_rung}")


def random_model(n: int, n_sys: int, seed: int, lam: float = 0.7, density: float = 0.6,
                 anisotropic: bool = True) -> ModelSpec:
    """Small random real model used to exercise every term kind in tests."""
    rng = np.random.default_rng(seed)
    jx, jy, jz, hz, gx = _empty(n)
    for a in range(n):
        for b in range(a + 1, n):
            if rng.random() < density:
                jx[a, b] = rng.normal()
                jy[a, b] = rng.normal() if anisotropic else jx[a, b]
                jz[a, b] = rng.normal()
    hz[:] = rng.normal(size=n) * 0.5
    gx[:] = rng.normal(size=n) * 0.5 if anisotropic else 0.0
    return ModelSpec(n, n_sys, jx, jy, jz, hz, gx, lam, f"random_N{n}_s{seed}")


def beta_grid(n: int, lo: float = 0.1, hi: float = 10.0) -> np.ndarray:
    """Geometric inverse-temperature grid including both ends."""
    if n == 1:
        return np.array([lo])
    return np.geomspace(lo, hi, n)


# ----------------------------------------------------------------------------
# The paper-shaped workloads (synthetic, seeded).
# ----------------------------------------------------------------------------

def config_c1():
    """XXZ periodic chain N=10, N_s=1, J=1, Delta=0.5, lambda=1, n_v=16, k=40."""
    spec = xxz_chain(10, 1, j=1.0, delta=0.5, h=0.0, lam=1.0, periodic=True)
    return dict(spec=spec, betas=np.array([0.5, 1.0, 2.0]), n_v=16, k=40,
                seed=20220417, dist="rademacher", precision="fp64")


def config_c2(g_index: int = 0):
    """Long-range TFIM N=22, alpha=1.5, N_s=2, g in linspace(0.2, 2, 16), n_v=32, k=60."""
    gs = np.linspace(0.2, 2.0, 16)
    spec = long_range_tfim(22, 2, alpha=1.5, g=float(gs[g_index]), lam=1.0)
    return dict(spec=spec, betas=np.array([1.0]), n_v=32, k=60,
                seed=20220418 + g_index, dist="gauss", precision="fp32")


def config_c3():
    """Long-range XXZ N=25, alpha=1, Delta=1, h=0.1, N_s=1, n_v=64, k=80, 32 betas."""
    spec = long_range_xxz(25, 1, alpha=1.0, delta=1.0, h=0.1, lam=1.0)
    return dict(spec=spec, betas=beta_grid(32, 0.1, 10.0), n_v=64, k=80,
                seed=20220420, dist="rademacher", precision="fp32")


def config_c5():
    """Long-range XXZ N=30, alpha=1.5, Delta=0.5, N_s=1, n_v=4, k=50, beta=2."""
    spec = long_range_xxz(30, 1, alpha=1.5, delta=0.5, h=0.0, lam=1.0)
    return dict(spec=spec, betas=np.array([2.0]), n_v=4, k=50,
                seed=20220421, dist="rademacher", precision="fp32")


def serving_requests(n_requests: int = 2000, seed: int = 20220419, n_min: int = 12,
                     n_max: int = 22):
    """Mixed request stream (XXZ or long-range TFIM, uneven N, beta grids, n_v, k).

    Returns a list of dicts with ``spec``, ``betas``, ``n_v``, ``k``, ``seed`` and
    the inter-arrival gap (exponential, unit mean; the caller scales it).
    """
    rng = np.random.default_rng(seed)
    out = []
    for r in range(n_requests):
        n = int(rng.integers(n_min, n_max + 1))
        n_sys = int(rng.integers(1, 3))
        lam = float(rng.uniform(0.1, 2.0))
        if rng.random() < 0.5:
            delta = float(rng.uniform(0.0, 2.0))
            alpha = [1.0, 1.5, math.inf][int(rng.integers(0, 3))]
            h = float(rng.uniform(0.0, 0.5))
            if math.isinf(alpha):
                spec = xxz_chain(n, n_sys, 1.0, delta, h, lam, periodic=False)
            else:
                spec = long_range_xxz(n, n_sys, alpha, delta, h, lam)
        else:
            g = float(rng.uniform(0.2, 2.0))
            spec = long_range_tfim(n, n_sys, 1.5, g, lam)
        n_beta = int(rng.integers(8, 65))
        out.append(dict(spec=spec, betas=beta_grid(n_beta, 0.1, 10.0),
                        n_v=int(rng.choice([8, 16, 32, 64])),
                        k=int(rng.integers(30, 101)),
                        seed=int(seed * 4096 + r),
                        gap=float(rng.exponential(1.0))))
    return out
