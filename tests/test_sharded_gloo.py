"""The host side of the bath-vector sharding over ranks: world_size-2 gloo on CPU.

Each rank computes its share of one estimate (here with the oracle, the CPU
stand-in for its GPU), the parts cross ranks through torch.distributed, and the
combined rho*, ln Z_t and E0 must equal the single-run oracle result.
"""
import os
import socket

import numpy as np
import pytest

import workloads as W


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _oracle_part(spec, betas, n_v, k, seed, dist, rank, world):
    from oracle import lanczos
    from paper_2204_08147_gb300.sharded import shard_range
    first, count = shard_range(n_v, rank, world)
    if count == 0:
        return dict(count=0, e0=np.inf, gram=None, quad=None)
    out = lanczos.Estimator(spec).run(betas, n_v, k, seed, dist, vectors=range(first, first + count))
    return dict(count=count, e0=out["e0"], gram=out["gram_l"].sum(axis=1), quad=out["quad_l"].sum(axis=1))


def _worker(rank, world, port, n_v, result_path):
    import torch.distributed as dist
    from paper_2204_08147_gb300.sharded import combine, gather_parts
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        spec = W.random_model(7, 1, 61)
        betas = np.array([0.4, 1.5, 4.0])
        part = _oracle_part(spec, betas, n_v, 12, 99, "gauss", rank, world)
        res = combine(gather_parts(part), betas, spec.d_b, n_v)
        if rank == 0:
            np.savez(result_path, **{k: np.asarray(v) for k, v in res.items()})
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("n_v", [5, 1])
def test_two_rank_combine_equals_single_run(tmp_path, n_v):
    import torch.multiprocessing as mp
    from oracle import lanczos
    path = str(tmp_path / "res.npz")
    mp.spawn(_worker, args=(2, _free_port(), n_v, path), nprocs=2, join=True)
    got = np.load(path)
    spec = W.random_model(7, 1, 61)
    betas = np.array([0.4, 1.5, 4.0])
    ref = lanczos.Estimator(spec).run(betas, n_v, 12, 99, "gauss")
    assert abs(float(got["e0"]) - ref["e0"]) < 1e-12
    np.testing.assert_allclose(got["rho"], ref["rho"], atol=1e-13)
    np.testing.assert_allclose(got["rho_quad"], ref["rho_quad"], atol=1e-13)
    np.testing.assert_allclose(got["lnZ"], ref["lnZ"], atol=1e-12)


def test_shard_ranges_cover_once():
    from paper_2204_08147_gb300.sharded import shard_range
    for n_v in (1, 7, 32, 33):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                f, c = shard_range(n_v, r, world)
                seen.extend(range(f, f + c))
            assert seen == list(range(n_v))


def test_combine_rejects_incomplete_parts():
    from paper_2204_08147_gb300.sharded import combine
    part = dict(count=2, e0=0.0, gram=np.ones((1, 2, 2)), quad=np.ones((1, 2, 2)))
    with pytest.raises(ValueError):
        combine([part], [1.0], 4, 3)
