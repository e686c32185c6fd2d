"""The all-to-all benchmark configurations at full size: sampled rows of H x.

c3 (long-range XXZ, N = 25, N_s = 1, h = 0.1) and c5 (N = 30, alpha = 1.5, Delta = 0.5)
are too large for the oracle's whole-vector SpMM. Their apply through the C ABI
(rdm_apply_hamiltonian: the tiled SpMM with the estimator's tile walk, partner tiles of
one high spin consumed in opposite-spin pairs and flat partner tiles) runs on a seeded
random block of 32-byte rows (8 float32 or 4 float64 columns) at the full 2^N states,
and 64 sampled rows are checked against the oracle's single-row construction (the
Pauli terms applied to one basis vector; eq. Ht, Sec. 2.2). Tolerance: a fixed multiple
of the working precision times sum_s' |H_ss'| |x_s'| of the row (float32 coefficients
and sums: 2e-5; float64: 1e-13); one missing or wrong term moves a row by about
1/(number of terms) of that sum.
"""
import numpy as np
import pytest

import workloads as W
from oracle import spin_ops

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


@pytest.mark.parametrize("config", ["c3", "c5"])
@pytest.mark.parametrize("dtype,ncols,tol", [("float32", 8, 2e-5), ("float64", 4, 1e-13)])
def test_full_size_apply_sampled_rows(lib, config, dtype, ncols, tol):
    torch = _torch()
    spec = (W.config_c3() if config == "c3" else W.config_c5())["spec"]
    d = 1 << spec.n_sites
    torch.cuda.empty_cache()  # blocks cached by earlier tests
    ctx = lib.Context(0)
    try:
        ham = lib.Hamiltonian(ctx, spec)
        gen = torch.Generator(device="cuda").manual_seed(20220425)
        x = torch.randn(d, ncols, dtype=getattr(torch, dtype), device="cuda", generator=gen)
        y = torch.empty_like(x)
        ham.apply(x, y)
        torch.cuda.synchronize()
        rng = np.random.default_rng(spec.n_sites)
        states = rng.integers(0, d, size=64)
        rows = [spin_ops.hamiltonian_row(spec, int(s)) for s in states]
        cols = np.concatenate([np.fromiter(r.keys(), dtype=np.int64) for r in rows])
        xs = x[torch.from_numpy(cols).cuda()].double().cpu().numpy()
        got = y[torch.from_numpy(states.astype(np.int64)).cuda()].double().cpu().numpy()
        at = 0
        for i, r in enumerate(rows):
            vals = np.fromiter(r.values(), dtype=np.float64)
            xr = xs[at:at + len(vals)]
            at += len(vals)
            want = vals @ xr
            scale = np.abs(vals) @ np.abs(xr)
            assert np.all(np.abs(got[i] - want) <= tol * scale), (config, dtype, int(states[i]))
        del x, y
        ham.close()
    finally:
        ctx.close()
        torch.cuda.empty_cache()
