"""The allocation-free starting block (rdm_starting_block_noalloc) against
rdm_starting_block, through the C ABI, on two calls in a row.

It serves callers that may not allocate device memory themselves (a framework
allocator that owns the memory budget, or loops where cudaMalloc/cudaFree would
synchronise the device). This file is collected last on purpose.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dist", ["gauss", "rademacher"])
def test_noalloc_starting_block_matches_allocating_entry_point(lib, dist):
    import torch
    ctx = lib.Context(0)
    try:
        spec = W.random_model(10, 2, 7)
        ham = lib.Hamiltonian(ctx, spec)
        n_v = 4
        for dtype, rtol in ((torch.float64, 4e-15), (torch.float32, 1.2e-7)):
            # two calls in a row with different seeds: the shared scratch must not leak
            for seed in (11, 12):
                ref = torch.empty((1 << 10, 4 * n_v), dtype=dtype, device="cuda")
                got = torch.full_like(ref, float("nan"))
                ham.starting_block(ref, n_v, seed, dist)
                ham.starting_block_noalloc(got, n_v, seed, dist)
                torch.cuda.synchronize()
                np.testing.assert_allclose(got.cpu().numpy(), ref.cpu().numpy(), rtol=rtol, atol=0)
        # beyond the scratch's 32 vectors
        big = torch.empty((1 << 10, 4 * 64), dtype=torch.float32, device="cuda")
        with pytest.raises(lib.RdmError) as e:
            ham.starting_block_noalloc(big, 64, 1, dist)
        assert e.value.status == lib.EINVAL and "maximum" in str(e.value)
        # within the scratch but beyond the column rule (float64, 4 * 8 = 32 > 16 columns)
        wide = torch.empty((1 << 10, 4 * 8), dtype=torch.float64, device="cuda")
        with pytest.raises(lib.RdmError) as e:
            ham.starting_block_noalloc(wide, 8, 1, dist)
        assert e.value.status == lib.EINVAL and "columns" in str(e.value)
        ham.close()
    finally:
        ctx.close()
