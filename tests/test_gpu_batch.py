"""rdm_estimate_batch: uneven instances whose first passes share one persistent launch.

The estimator is a sum of independent recurrences (Sec. 3.1), so estimates of several
Hamiltonians can run side by side. Checks, through the C ABI:
  * every item of a mixed batch (different N, N_s, n_v, k, betas, precisions, vector
    distributions) matches the oracle (float64: 1e-10, float32: 1e-4 on rho*), and
    the same estimate run on its own through rdm_estimate (float64 items that take the
    untiled kernels: bit-identical; others within the precision contract);
  * an item's result is bit-identical alone (a batch of one) and in the mix;
  * the autotuner times its candidates once per size class and reuses the choice;
  * items the packed launch does not take (recomputed basis) run alongside.
"""
import numpy as np
import pytest

import workloads as W
from oracle import lanczos

pytestmark = pytest.mark.gpu


def _jobs(lib, ctx):
    specs = [
        (W.random_model(8, 2, 11), dict(n_v=3, k=12, seed=5, precision="fp64", dist="rademacher",
                                        betas=[0.5, 1.0])),
        (W.xxz_chain(10, 1, 1.0, 0.5), dict(n_v=16, k=40, seed=20220417, precision="fp64",
                                           dist="rademacher", betas=[0.5, 1.0, 2.0])),
        (W.long_range_tfim(11, 2, 1.5, 0.9), dict(n_v=5, k=25, seed=7, precision="fp32", dist="gauss",
                                                  betas=[1.0])),
        (W.random_model(9, 1, 3), dict(n_v=7, k=18, seed=9, precision="fp32", dist="rademacher",
                                       betas=[0.3, 3.0])),
        (W.long_range_xxz(12, 1, 1.0, 1.0, 0.1), dict(n_v=8, k=30, seed=13, precision="fp32",
                                                      dist="rademacher", betas=[0.7])),
        (W.random_model(7, 2, 4), dict(n_v=2, k=9, seed=17, precision="fp64", dist="gauss",
                                       betas=[1.5])),
    ]
    jobs = []
    for spec, kw in specs:
        jb = dict(kw)
        jb["ham"] = lib.Hamiltonian(ctx, spec)
        jb["spec"] = spec
        jobs.append(jb)
    return jobs


def test_batch_matches_oracle_and_single_estimates(lib):
    ctx = lib.Context(0)
    try:
        jobs = _jobs(lib, ctx)
        outs = ctx.estimate_batch(jobs)
        for jb, out in zip(jobs, outs):
            assert out["status"] == lib.OK
            tol = 1e-10 if jb["precision"] == "fp64" else 1e-4
            ref = lanczos.Estimator(jb["spec"]).run(jb["betas"], jb["n_v"], jb["k"], jb["seed"], jb["dist"])
            np.testing.assert_allclose(out["rho"], ref["rho"], atol=tol, rtol=0)
            single = jb["ham"].estimate(jb["betas"], jb["n_v"], jb["k"], jb["seed"], precision=jb["precision"],
                                        dist=jb["dist"])
            np.testing.assert_allclose(out["rho"], single["rho"], atol=tol, rtol=0)
            np.testing.assert_allclose(out["lnZ"], single["lnZ"], atol=1e3 * tol, rtol=0)
            if jb["precision"] == "fp64" and jb["spec"].n_sites < 10:  # both untiled: same arithmetic
                np.testing.assert_array_equal(out["rho"], single["rho"])
    finally:
        ctx.close()


def test_batch_item_alone_equals_in_mix(lib):
    ctx = lib.Context(0)
    try:
        jobs = _jobs(lib, ctx)
        mix = ctx.estimate_batch(jobs, full=True)
        for jb, m in zip(jobs, mix):
            alone = ctx.estimate_batch([jb], full=True)[0]
            for key in ("rho", "lnZ", "gram_l", "t_a", "t_b"):
                np.testing.assert_array_equal(alone[key], m[key])
        # order of the items in the batch does not matter either
        rev = ctx.estimate_batch(jobs[::-1])
        for a, b in zip(rev[::-1], mix):
            np.testing.assert_array_equal(a["rho"], b["rho"])
    finally:
        ctx.close()


def test_batch_autotuner_times_each_size_class_once(lib):
    ctx = lib.Context(0)
    try:
        jobs = _jobs(lib, ctx)
        assert ctx.packed_tuning() == (0, 0)
        ctx.estimate_batch(jobs)
        keys, runs = ctx.packed_tuning()
        assert keys >= 1 and runs >= keys
        ctx.estimate_batch(jobs)
        assert ctx.packed_tuning() == (keys, runs)
    finally:
        ctx.close()


def test_batch_with_items_outside_the_packed_launch(lib):
    ctx = lib.Context(0)
    try:
        jobs = _jobs(lib, ctx)[:3]
        jobs[1] = dict(jobs[1], passes="recompute")  # recomputed basis: runs as rdm_estimate does
        outs = ctx.estimate_batch(jobs)
        for jb, out in zip(jobs, outs):
            single = jb["ham"].estimate(jb["betas"], jb["n_v"], jb["k"], jb["seed"], precision=jb["precision"],
                                        dist=jb["dist"], passes=jb.get("passes", "auto"))
            tol = 1e-10 if jb["precision"] == "fp64" else 1e-4
            np.testing.assert_allclose(out["rho"], single["rho"], atol=tol, rtol=0)
    finally:
        ctx.close()


def test_batch_rejects_a_foreign_hamiltonian(lib):
    a, b = lib.Context(0), lib.Context(0)
    try:
        ham = lib.Hamiltonian(b, W.random_model(6, 1, 2))
        with pytest.raises(lib.RdmError) as e:
            a.estimate_batch([dict(ham=ham, betas=[1.0], n_v=2, k=4, seed=1)])
        assert e.value.status == lib.EINVAL
    finally:
        a.close()
        b.close()


def test_batch_device_dense_steps_in_one_launch(lib):
    """Items with 10-point beta grids take the device small dense step; a batch runs all
    their recurrences (both d_s groups) in one launch per d_s. Against each estimate on
    its own with the host path: float64 items within 1e-12 in rho*, float32 within the
    float32 contract."""
    ctx = lib.Context(0)
    try:
        jobs = _jobs(lib, ctx)
        for jb in jobs:
            jb["betas"] = list(W.beta_grid(10, 0.2, 6.0))
        ctx.profile(True)
        outs = ctx.estimate_batch(jobs)
        st = ctx.profile_stats()
        ctx.profile(False)
        assert st["dense_fT"]["launches"] == 2  # d_s = 2 and d_s = 4 groups
        ctx.set_device_dense(0)
        for jb, out in zip(jobs, outs):
            single = jb["ham"].estimate(jb["betas"], jb["n_v"], jb["k"], jb["seed"], precision=jb["precision"],
                                        dist=jb["dist"])
            tol = 1e-12 if jb["precision"] == "fp64" else 1e-4
            np.testing.assert_allclose(out["rho"], single["rho"], atol=tol, rtol=0)
    finally:
        ctx.close()


def test_batch_launch_forms_are_bit_identical(lib):
    """The packed first pass as the cooperative grid (grid barriers between phases) and
    as one block per slice (block barriers only): the same units with the same arithmetic,
    so every item's result is the same bit for bit; an unknown form is rejected."""
    ctx = lib.Context(0)
    try:
        jobs = _jobs(lib, ctx)
        outs = {}
        for form in (1, 2):
            ctx.set_packed_form(form)
            outs[form] = ctx.estimate_batch(jobs, full=True)
        for a, b in zip(outs[1], outs[2]):
            for key in ("rho", "lnZ", "gram_l", "t_a", "t_b"):
                np.testing.assert_array_equal(a[key], b[key])
        with pytest.raises(lib.RdmError) as e:
            ctx.set_packed_form(3)
        assert e.value.status == lib.EINVAL
    finally:
        ctx.close()
