"""One estimate split over ranks by bath vectors (one GPU per rank).

The estimator is a sum over bath vectors (eq. trace_est, eq. trB_est), so rank r runs
vectors [first_r, first_r + n_r) of the same seeded sequence through the library and
only two things cross ranks, on the host: the shift E0 = min over ranks of E0_r
(Sec. 3.2) and the d_s x d_s Gram sums. A rank's sums are relative to its own
shift, S_r(beta) = sum_{l in r} G_l(E0_r); the total is
    S(beta) = sum_r exp(-beta (E0_r - E0)) S_r(beta),
folded in rank order, then normalised as eq. rho_est with
ln Z_t = ln(d_b tr S / n_v) - beta E0.
"""
from __future__ import annotations

import numpy as np


def shard_range(n_v: int, rank: int, world: int):
    """(first, count) of rank's bath vectors: contiguous, sizes differ by at most 1."""
    base, extra = divmod(n_v, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def local_part(ham, betas, n_v, k, seed, rank, world, **estimate_kw) -> dict:
    """Runs this rank's share of the bath vectors on its GPU and returns its sums."""
    first, count = shard_range(n_v, rank, world)
    betas = np.atleast_1d(np.asarray(betas, dtype=np.float64))
    if count == 0:
        return dict(count=0, e0=np.inf, gram=None, quad=None)
    out = ham.estimate(betas, count, k, seed, full=True, first_vector=first, **estimate_kw)
    return dict(count=count, e0=float(out["e0"]), gram=out["gram_l"].sum(axis=1),
                quad=out["quad_l"].sum(axis=1))


def combine(parts, betas, d_b: int, n_v: int) -> dict:
    """Folds per-rank sums (in the given rank order) into rho*, ln Z_t and E0."""
    betas = np.atleast_1d(np.asarray(betas, dtype=np.float64))
    live = [p for p in parts if p["count"] > 0]
    if sum(p["count"] for p in live) != n_v:
        raise ValueError("the parts do not cover every bath vector exactly once")
    e0 = min(p["e0"] for p in live)
    out = dict(e0=e0)
    for key, name in (("gram", "rho"), ("quad", "rho_quad")):
        tot = None
        for p in live:
            scale = np.exp(-betas * (p["e0"] - e0))[:, None, None]
            term = scale * p[key]
            tot = term if tot is None else tot + term
        tr = np.trace(tot, axis1=1, axis2=2)
        rho = tot / tr[:, None, None]
        out[name] = 0.5 * (rho + np.swapaxes(rho, 1, 2))
        if key == "gram":
            out["lnZ"] = np.log(d_b * tr / n_v) - betas * e0
    return out


def gather_parts(part: dict, group=None) -> list:
    """All ranks' parts, in rank order, through torch.distributed (any backend)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, part, group=group)
    return parts


def estimate_sharded(ham, betas, n_v, k, seed, group=None, **estimate_kw) -> dict:
    """rho*, ln Z_t of one run whose bath vectors are spread over the group's ranks."""
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    part = local_part(ham, betas, n_v, k, seed, rank, world, **estimate_kw)
    d_b = 1 << (int(ham.n_sites) - int(ham.n_sys))
    return combine(gather_parts(part, group), betas, d_b, n_v)
