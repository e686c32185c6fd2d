"""Parity of the CUDA path (through the C ABI) against the CPU oracle.

Tolerances: the SpMM index logic is bit-exact (integer-valued data in float64 makes
every sum exact); rho* entries within 1e-10 (float64 path) or 1e-4 (float32 path)
max-abs of the oracle on the same seeded bath vectors.
"""
import numpy as np
import pytest

import workloads as W
from oracle import closed_form, exact, lanczos, post, rng as orng, spin_ops

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-4


@pytest.fixture(scope="module")
def ctx(lib):
    """A context whose estimates take the tiled SpMM wherever the layout allows it (the
    small test problems would otherwise run the plain kernel, which the default form
    picks below 32 tiles), so the estimator's tiled modes are checked at every size."""
    c = lib.Context(0)
    c.set_spmm_form(1)
    yield c
    c.close()


def _torch():
    import torch
    return torch


# ---------------------------------------------------------------- a1 + a3: SpMM

def _integer_model(n, n_sys, seed, lam=1.0):
    r = np.random.default_rng(seed)
    spec = W.random_model(n, n_sys, seed, lam=lam)
    for t in (spec.jx, spec.jy, spec.jz):
        t[:] = np.round(t * 2)
    spec.hz[:] = np.round(spec.hz * 4)
    spec.gx[:] = np.round(spec.gx * 4)
    del r
    return spec


@pytest.mark.parametrize("n,n_sys,seed", [(2, 1, 1), (5, 0, 2), (7, 1, 3), (9, 2, 4), (11, 1, 5)])
@pytest.mark.parametrize("ncols", [2, 8, 16])
def test_apply_bit_exact_index_logic_fp64(ctx, lib, n, n_sys, seed, ncols):
    torch = _torch()
    spec = _integer_model(n, n_sys, seed, lam=2.0)
    h = spin_ops.dense_hamiltonian(spec)
    x = np.random.default_rng(seed).integers(-3, 4, size=(1 << n, ncols)).astype(np.float64)
    ham = lib.Hamiltonian(ctx, spec)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    ham.apply(xd, yd)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(yd.cpu().numpy(), h @ x)


@pytest.mark.parametrize("n,n_sys,seed", [(10, 1, 20), (11, 1, 21), (12, 2, 22), (13, 0, 23), (15, 1, 24)])
@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_apply_tiled_bit_exact(ctx, lib, n, n_sys, seed, dtype):
    """A 32-byte row per state (8 float32 / 4 float64 columns, N >= 10) takes the
    tiled SpMM: 1024-state tiles, partner tiles by bulk copies, the diagonal rebuilt
    per tile from its low-bit table and row-group coefficients. Integer couplings and
    inputs make every sum exact, so the result must equal H x bit for bit."""
    torch = _torch()
    spec = _integer_model(n, n_sys, seed, lam=2.0)
    h = spin_ops.sparse_hamiltonian(spec)
    ncols = 8 if dtype == "float32" else 4
    x = np.random.default_rng(seed).integers(-3, 4, size=(1 << n, ncols)).astype(np.float64)
    ham = lib.Hamiltonian(ctx, spec)
    xd = torch.from_numpy(x).to(getattr(torch, dtype)).cuda()
    yd = torch.empty_like(xd)
    ham.apply(xd, yd)
    ham.apply(xd, yd)  # second call reuses the Hamiltonian's tile table
    torch.cuda.synchronize()
    np.testing.assert_array_equal(yd.double().cpu().numpy(), h @ x)


@pytest.mark.parametrize("n,n_sys,seed", [(6, 1, 11), (10, 2, 12), (12, 0, 13)])
@pytest.mark.parametrize("ncols,dtype", [(4, "float32"), (32, "float32"), (2, "float64"), (16, "float64")])
def test_apply_real_couplings(ctx, lib, n, n_sys, seed, ncols, dtype):
    torch = _torch()
    spec = W.random_model(n, n_sys, seed)
    h = spin_ops.dense_hamiltonian(spec)
    x = np.random.default_rng(seed).normal(size=(1 << n, ncols))
    ham = lib.Hamiltonian(ctx, spec)
    tdt = getattr(torch, dtype)
    xd = torch.from_numpy(x).to(tdt).cuda()
    yd = torch.empty_like(xd)
    ham.apply(xd, yd)
    torch.cuda.synchronize()
    ref = h @ xd.double().cpu().numpy()
    tol = 1e-13 if dtype == "float64" else 1e-5
    scale = np.abs(h).sum(axis=1).max() * np.abs(x).max()
    assert np.abs(yd.double().cpu().numpy() - ref).max() <= tol * scale


def test_apply_rejects_bad_columns(ctx, lib):
    torch = _torch()
    ham = lib.Hamiltonian(ctx, W.random_model(4, 1, 1))
    x = torch.zeros((16, 6), dtype=torch.float32, device="cuda")
    with pytest.raises(lib.RdmError) as e:
        ham.apply(x, torch.zeros_like(x))
    assert e.value.status == lib.EINVAL


# ---------------------------------------------------------------- a2: starting block

@pytest.mark.parametrize("dist", ["rademacher", "gauss", "basis"])
@pytest.mark.parametrize("n,n_sys,n_v", [(8, 1, 4), (9, 2, 4), (10, 0, 8)])
def test_starting_block_matches_generator(ctx, lib, dist, n, n_sys, n_v):
    torch = _torch()
    spec = W.random_model(n, n_sys, 3)
    ham = lib.Hamiltonian(ctx, spec)
    d_s = 1 << n_sys
    ref = np.hstack([orng.starting_block(d_s, orng.bath_vector(spec.d_b, l, 1234, dist)) for l in range(n_v)])
    for dtype in ("float64", "float32"):
        x = torch.empty((1 << n, d_s * n_v), dtype=getattr(torch, dtype), device="cuda")
        ham.starting_block(x, n_v, 1234, dist)
        torch.cuda.synchronize()
        got = x.cpu().numpy()
        want = ref.astype(dtype)
        if dist == "gauss":
            np.testing.assert_allclose(got, want, rtol=4e-15 if dtype == "float64" else 1.2e-7, atol=0)
        else:
            np.testing.assert_array_equal(got, want)


# ---------------------------------------------------------------- a4: recurrence

def test_lanczos_coefficients_match_oracle_fp64(ctx, lib):
    spec = W.random_model(9, 2, 21)
    ham = lib.Hamiltonian(ctx, spec)
    k = 6
    out = ham.estimate([1.0], n_v=3, k=k, seed=5, precision="fp64", dist="rademacher", full=True)
    est = lanczos.Estimator(spec)
    for l in range(3):
        a_l, b_l = lanczos.lanczos_coefficients(est.apply_h, est.starting_block(l, 5, "rademacher"), k, est.hnorm)
        np.testing.assert_allclose(out["t_a"][l], np.array(a_l), atol=1e-12)
        np.testing.assert_allclose(out["t_b"][l], np.array(b_l), atol=1e-12)
        for b in out["t_b"][l]:
            assert np.all(np.tril(b, -1) == 0) and np.all(np.diag(b) >= 0)


# ---------------------------------------------------------------- full estimator

def test_c1_fp64_matches_oracle(ctx, lib):
    c = W.config_c1()
    ham = lib.Hamiltonian(ctx, c["spec"])
    out = ham.estimate(c["betas"], c["n_v"], c["k"], c["seed"], precision="fp64", dist=c["dist"], full=True)
    ref = lanczos.Estimator(c["spec"]).run(c["betas"], c["n_v"], c["k"], c["seed"], c["dist"])
    assert abs(out["e0"] - ref["e0"]) < 1e-10
    np.testing.assert_allclose(out["rho"], ref["rho"], atol=TOL64, rtol=0)
    np.testing.assert_allclose(out["rho_quad"], ref["rho_quad"], atol=TOL64, rtol=0)
    np.testing.assert_allclose(out["lnZ"], ref["lnZ"], atol=1e-9, rtol=0)
    np.testing.assert_allclose(out["gram_l"], ref["gram_l"], atol=1e-10 * np.abs(ref["gram_l"]).max())


def test_c1_fp32_matches_oracle(ctx, lib):
    c = W.config_c1()
    ham = lib.Hamiltonian(ctx, c["spec"])
    out = ham.estimate(c["betas"], c["n_v"], c["k"], c["seed"], precision="fp32", dist=c["dist"])
    ref = lanczos.Estimator(c["spec"]).run(c["betas"], c["n_v"], c["k"], c["seed"], c["dist"])
    np.testing.assert_allclose(out["rho"], ref["rho"], atol=TOL32, rtol=0)
    np.testing.assert_allclose(out["lnZ"], ref["lnZ"], atol=1e-3, rtol=0)


@pytest.mark.parametrize("n,n_sys", [(7, 1), (8, 2), (6, 0)])
def test_exhaustive_basis_equals_exact_partial_trace(ctx, lib, n, n_sys):
    spec = W.random_model(n, n_sys, 40 + n)
    betas = [0.0, 0.3, 1.0, 4.0]
    ham = lib.Hamiltonian(ctx, spec)
    k = (1 << n) // spec.d_s + 2
    out = ham.estimate(betas, spec.d_b, k, 0, precision="fp64", dist="basis")
    rho, lnz = exact.exact_rho(spec, betas)
    np.testing.assert_allclose(out["rho"], rho, atol=TOL64, rtol=0)
    np.testing.assert_allclose(out["rho_quad"], rho, atol=TOL64, rtol=0)
    np.testing.assert_allclose(out["lnZ"], lnz, atol=1e-9, rtol=0)


def test_xy_chain_matches_app_c_closed_form(ctx, lib):
    n = 8
    spec = W.xy_open_chain(n, 2, 1.0, 0.3)
    betas = np.geomspace(0.1, 10.0, 7)
    ham = lib.Hamiltonian(ctx, spec)
    out = ham.estimate(betas, spec.d_b, 70, 0, precision="fp64", dist="basis")
    for i, beta in enumerate(betas):
        np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(out["rho"][i])),
                                   closed_form.rho_eigenvalues(n, beta, 1.0, 0.3), atol=TOL64)
        assert abs(out["lnZ"][i] - closed_form.log_partition_chain(n, beta, 1.0, 0.3)) < 1e-9


def test_uncoupled_model_gives_bare_system_gibbs(ctx, lib):
    spec = W.random_model(10, 2, 50, lam=0.0)
    ham = lib.Hamiltonian(ctx, spec)
    out = ham.estimate([0.5, 2.0], 3, 60, 9, precision="fp64", dist="gauss")
    for i, beta in enumerate([0.5, 2.0]):
        np.testing.assert_allclose(out["rho"][i], exact.bare_system_gibbs(spec, beta), atol=TOL64)
    out32 = ham.estimate([0.5, 2.0], 3, 60, 9, precision="fp32", dist="gauss")
    for i, beta in enumerate([0.5, 2.0]):
        np.testing.assert_allclose(out32["rho"][i], exact.bare_system_gibbs(spec, beta), atol=TOL32)


def test_beta_zero_is_maximally_mixed(ctx, lib):
    spec = W.random_model(9, 2, 51)
    ham = lib.Hamiltonian(ctx, spec)
    for prec in ("fp64", "fp32"):
        out = ham.estimate([0.0], 4, 10, 3, precision=prec, dist="rademacher")
        np.testing.assert_allclose(out["rho"][0], np.eye(4) / 4, atol=1e-15 if prec == "fp64" else 1e-7)


def test_low_temperature_limit(ctx, lib):
    spec = W.random_model(8, 1, 13)
    solver = exact.ExactSolver(spec)
    beta = 40.0 / (solver.evals[1] - solver.evals[0])
    ham = lib.Hamiltonian(ctx, spec)
    out = ham.estimate([beta], spec.d_b, 160, 0, precision="fp64", dist="basis")
    np.testing.assert_allclose(out["rho"][0], solver.ground_state_reduced(), atol=1e-6)


@pytest.mark.parametrize("n_v,k", [(1, 1), (1, 7), (5, 12), (13, 20)])
def test_ragged_sizes_match_oracle(ctx, lib, n_v, k):
    spec = W.random_model(9, 1, 60 + n_v)
    ham = lib.Hamiltonian(ctx, spec)
    betas = [0.4, 1.7]
    out = ham.estimate(betas, n_v, k, 77, precision="fp64", dist="gauss", full=True)
    ref = lanczos.Estimator(spec).run(betas, n_v, k, 77, "gauss")
    np.testing.assert_allclose(out["rho"], ref["rho"], atol=TOL64)
    np.testing.assert_allclose(out["rho_quad"], ref["rho_quad"], atol=TOL64)
    out32 = ham.estimate(betas, n_v, k, 77, precision="fp32", dist="gauss")
    np.testing.assert_allclose(out32["rho"], ref["rho"], atol=TOL32)


def test_tiny_system_two_sites(ctx, lib):
    spec = W.xxz_chain(2, 1, 1.0, 0.5, 0.2, 1.0, periodic=False)
    ham = lib.Hamiltonian(ctx, spec)
    out = ham.estimate([1.0], 2, 3, 0, precision="fp64", dist="basis")
    rho, _ = exact.exact_rho(spec, [1.0])
    np.testing.assert_allclose(out["rho"], rho, atol=TOL64)


def test_deterministic_bitwise(ctx, lib):
    spec = W.long_range_tfim(14, 2, 1.5, 0.8)
    ham = lib.Hamiltonian(ctx, spec)
    a = ham.estimate([1.0, 2.0], 8, 30, 11, precision="fp32", dist="gauss", full=True)
    b = ham.estimate([1.0, 2.0], 8, 30, 11, precision="fp32", dist="gauss", full=True)
    for key in ("rho", "gram_l", "t_a", "t_b"):
        np.testing.assert_array_equal(a[key], b[key])


def test_post_processing_of_gpu_rho(ctx, lib):
    c = W.config_c1()
    ham = lib.Hamiltonian(ctx, c["spec"])
    out = ham.estimate(c["betas"], c["n_v"], c["k"], c["seed"], precision="fp64")
    for i, beta in enumerate(c["betas"]):
        np.testing.assert_allclose(lib.mean_force(out["rho"][i], beta), post.mean_force(out["rho"][i], beta), atol=1e-12)
        assert abs(lib.entropy(out["rho"][i]) - post.entropy(out["rho"][i])) < 1e-13


# ---------------------------------------------------------------- c2-shaped, FP32 vs FP64 oracle

@pytest.mark.parametrize("n,n_sys,n_v", [(12, 1, 6), (13, 0, 3), (12, 2, 5), (11, 2, 1)])
def test_tiled_fp64_estimate_vs_oracle(ctx, lib, n, n_sys, n_v):
    """float64 runs the tiled SpMM (32-byte slice rows); with d_s = 4 a bath vector's
    group of four columns is the whole row, split over the row's two 16-byte lanes.
    Every term kind of a random model against the oracle at the float64 tolerance."""
    spec = W.random_model(n, n_sys, 70 + n)
    betas = [0.2, 1.0, 3.0]
    ham = lib.Hamiltonian(ctx, spec)
    out = ham.estimate(betas, n_v, 30, 5, precision="fp64", dist="gauss")
    ref = lanczos.Estimator(spec).run(betas, n_v, 30, 5, "gauss")
    np.testing.assert_allclose(out["rho"], ref["rho"], atol=TOL64, rtol=0)
    np.testing.assert_allclose(out["lnZ"], ref["lnZ"], atol=1e-9, rtol=0)


def test_lr_tfim_small_fp32_vs_oracle(ctx, lib):
    spec = W.long_range_tfim(12, 2, 1.5, 1.1)
    ham = lib.Hamiltonian(ctx, spec)
    out = ham.estimate([1.0], 32, 60, 20220418, precision="fp32", dist="gauss", full=True)
    ref = lanczos.Estimator(spec).run([1.0], 32, 60, 20220418, "gauss")
    np.testing.assert_allclose(out["rho"], ref["rho"], atol=TOL32)
    assert abs(out["lnZ"][0] - ref["lnZ"][0]) < 1e-3


def test_c2_full_size_sampled_vector(ctx, lib):
    """Full-size LR-TFIM N=22 in the benchmark's launch configuration (n_v=32, k=60,
    float32): the first Lanczos coefficients of a sampled bath vector against the
    oracle run on that vector alone, plus properties of the whole result."""
    c = W.config_c2(0)
    ham = lib.Hamiltonian(ctx, c["spec"])
    out = ham.estimate(c["betas"], c["n_v"], c["k"], c["seed"], precision="fp32", dist=c["dist"], full=True)
    steps = 4
    for l in (0, 31):
        est = lanczos.Estimator(c["spec"])
        a_l, b_l = lanczos.lanczos_coefficients(est.apply_h, est.starting_block(l, c["seed"], c["dist"]),
                                                steps, est.hnorm)
        scale = est.hnorm
        assert np.abs(out["t_a"][l, :steps] - np.array(a_l)).max() < 2e-5 * scale
        assert np.abs(out["t_b"][l, :steps] - np.array(b_l)).max() < 2e-5 * scale
    rho = out["rho"][0]
    np.testing.assert_allclose(rho, rho.T, atol=1e-15)
    assert abs(np.trace(rho) - 1) < 1e-12 and np.linalg.eigvalsh(rho).min() > 0
    # Gram and quadrature forms agree while the float32 basis stays orthogonal enough.
    np.testing.assert_allclose(out["rho"], out["rho_quad"], atol=TOL32)
    # float32 against the float64 GPU path on the same seeds (the whole 32-vector sum).
    out64 = ham.estimate(c["betas"], c["n_v"], c["k"], c["seed"], precision="fp64", dist=c["dist"])
    np.testing.assert_allclose(out["rho"], out64["rho"], atol=TOL32)
    assert abs(out["lnZ"][0] - out64["lnZ"][0]) < 1e-3 * abs(out64["lnZ"][0])


# ---------------------------------------------------------------- serving

def test_serving_alone_equals_in_mix(ctx, lib):
    """Each request's result is the same whether it is served alone (submitted after the
    previous one finished) or in a mix that arrives at once (small requests then share
    packed launches), bit for bit; and it matches rdm_estimate run on its own within the
    float32 contract."""
    reqs = W.serving_requests(12, seed=5, n_min=8, n_max=14)
    for r in reqs:  # keep the host eigen-step of the test small
        r["n_v"] = min(r["n_v"], 16)
        r["k"] = min(r["k"], 40)
        r["betas"] = r["betas"][:12]
    ctx.serve_start(8 << 30, max_inflight=4)
    try:
        alone = []
        for r in reqs:
            t = ctx.submit(r["spec"], r["betas"], r["n_v"], r["k"], r["seed"], precision="fp32")
            alone.append(ctx.wait(t))
        tickets = [ctx.submit(r["spec"], r["betas"], r["n_v"], r["k"], r["seed"], precision="fp32") for r in reqs]
        for t, a in zip(tickets, alone):
            res = ctx.wait(t)
            np.testing.assert_array_equal(res["rho"], a["rho"])
            np.testing.assert_array_equal(res["lnZ"], a["lnZ"])
            lat, q = ctx.request_times(t)
            assert lat >= q >= 0
    finally:
        ctx.serve_stop()
    for r, a in zip(reqs, alone):
        ham = lib.Hamiltonian(ctx, r["spec"])
        single = ham.estimate(r["betas"], r["n_v"], r["k"], r["seed"], precision="fp32")
        ham.close()
        np.testing.assert_allclose(a["rho"], single["rho"], atol=TOL32, rtol=0)


# ---------------------------------------------------------------- copy-rate probe

def test_copy_rate_probe(ctx, lib):
    """The bulk-copy probe (the SpMM's on-chip roofline denominator) returns a finite
    rate with L2 no slower than DRAM, and rejects invalid arguments."""
    l2 = ctx.probe_copy_rate(32 << 20)
    dram = ctx.probe_copy_rate(1 << 30)
    assert 500.0 < dram < 100000.0 and 500.0 < l2 < 100000.0
    assert l2 > 0.9 * dram
    for bad in [(32 << 20, 0), (32 << 20, 9), (1 << 20, 6)]:
        with pytest.raises(lib.RdmError) as e:
            ctx.probe_copy_rate(*bad)
        assert e.value.status == lib.EINVAL


# ---------------------------------------------------------------- launch graphs

@pytest.mark.parametrize("case", ["c1_fp64", "tfim_fp32_tiled", "single_fp32"])
def test_graph_replay_is_bit_identical(ctx, lib, case):
    """The first pass replayed from a recorded CUDA graph (second and later calls of
    one configuration) gives the same bits as direct launches; a call with another
    configuration in between neither replays the wrong graph nor disturbs it."""
    if case == "c1_fp64":
        c = W.config_c1()
        spec, betas, n_v, k, seed, prec, dist, rec = c["spec"], c["betas"], c["n_v"], c["k"], c["seed"], \
            "fp64", c["dist"], "block"
    elif case == "tfim_fp32_tiled":
        spec, betas, n_v, k, seed, prec, dist, rec = W.long_range_tfim(12, 2, 1.5, 0.9), [0.5, 2.0], 8, 25, \
            11, "fp32", "gauss", "block"
    else:
        spec, betas, n_v, k, seed, prec, dist, rec = W.random_model(11, 2, 41), [1.0], 4, 12, 5, "fp32", \
            "gauss", "single"
    ham = lib.Hamiltonian(ctx, spec)

    def run(kk):
        return ham.estimate(betas, n_v, kk, seed, precision=prec, dist=dist, full=True, recurrence=rec)
    keys = ("rho", "lnZ", "gram_l", "quad_l", "t_a", "t_b")
    try:
        ctx.set_graphs(False)
        ref, ref2 = run(k), run(k + 3)
        ctx.set_graphs(True)
        outs = [run(k), run(k), run(k), run(k + 3), run(k), run(k + 3), run(k + 3)]
    finally:
        ctx.set_graphs(True)
        ham.close()
    for o, r in zip(outs, [ref, ref, ref, ref2, ref, ref2, ref2]):
        for key in keys:
            np.testing.assert_array_equal(o[key], r[key])


# ---------------------------------------------------------------- storage modes

def test_store_and_recompute_are_bit_identical(ctx, lib):
    spec = W.long_range_tfim(14, 2, 1.5, 0.7)
    ham = lib.Hamiltonian(ctx, spec)
    betas = [0.3, 1.0, 2.5, 6.0, 9.0]
    for prec in ("fp32", "fp64"):
        a = ham.estimate(betas, 8, 30, 4, precision=prec, dist="gauss", full=True, passes="store")
        b = ham.estimate(betas, 8, 30, 4, precision=prec, dist="gauss", full=True, passes="recompute")
        for key in ("rho", "lnZ", "gram_l", "quad_l", "t_a", "t_b"):
            np.testing.assert_array_equal(a[key], b[key])


def test_beta_chunks_in_a_small_workspace(ctx, lib):
    """A caller workspace that holds one psi block forces one pass-2 sweep per beta."""
    spec = W.long_range_xxz(13, 1, 1.0, 1.0, 0.1)
    ham = lib.Hamiltonian(ctx, spec)
    betas = list(W.beta_grid(5, 0.1, 10.0))
    ref = ham.estimate(betas, 16, 25, 8, precision="fp32", dist="rademacher", full=True, passes="store")
    nbytes = ham.workspace_size(len(betas), 16, 25, precision="fp32", dist="rademacher")
    ctx.attach_workspace(nbytes)
    try:
        got = ham.estimate(betas, 16, 25, 8, precision="fp32", dist="rademacher", full=True, passes="recompute")
    finally:
        ctx.detach_workspace()
    for key in ("rho", "lnZ", "gram_l"):
        np.testing.assert_array_equal(got[key], ref[key])
    with pytest.raises(lib.RdmError) as e:  # storing every block does not fit that workspace
        ctx.attach_workspace(nbytes)
        try:
            ham.estimate(betas, 16, 25, 8, precision="fp32", passes="store")
        finally:
            ctx.detach_workspace()
    assert e.value.status == lib.ENOMEM


@pytest.mark.parametrize("n_sys,n_v,prec,dist", [(1, 16, "fp32", "rademacher"), (1, 14, "fp32", "gauss"),
                                                 (1, 13, "fp64", "gauss"), (2, 7, "fp32", "gauss"),
                                                 (2, 5, "fp64", "rademacher")])
def test_slice_sweeps_when_psi_of_all_betas_fits_some_slices(ctx, lib, n_sys, n_v, prec, dist):
    """Caller workspaces from the default size down to the smallest that runs, in
    eighths of a block: where psi of every beta fits over some of the block's slices
    (32-byte rows: 4 bath vectors of d_s = 2 per float32 slice, 2 per float64 slice) but
    not over all, pass 2 sweeps over groups of slices with every beta; below that, over
    groups of betas at full width. Every size gives the stored-basis result bit for bit,
    and the slice sweeps run fewer pass-2 SpMM bytes than the beta sweeps (no recurrence
    repeated). Also with a padded last slice (n_v = 14, 13, 7), Gaussian vectors (each
    slice group reads its own rows of the generated vectors) and d_s = 4 (float64: one
    bath vector fills a row). The mode is read from the
    psi_init launches: slice sweeps write (1 + n_beta) blocks in all, beta sweeps one
    more block per extra sweep."""
    spec = W.long_range_xxz(13, n_sys, 1.0, 1.0, 0.1)
    ham = lib.Hamiltonian(ctx, spec)
    # more betas than slices, so that below some size psi of every beta over one slice
    # no longer fits while one beta's at full width does; the small dense step on the
    # host throughout (a small workspace would otherwise drop the device step's arrays
    # and change the coefficients' rounding)
    betas = list(W.beta_grid(9, 0.1, 10.0))
    ctx.set_device_dense(0)
    try:
        _slice_sweep_scan(ctx, lib, ham, betas, n_v, prec, dist, 1 << n_sys)
    finally:
        ctx.set_device_dense(1)


def _slice_sweep_scan(ctx, lib, ham, betas, n_v, prec, dist, d_s):
    ref = ham.estimate(betas, n_v, 25, 8, precision=prec, dist=dist, full=True, passes="store")
    nbytes = ham.workspace_size(len(betas), n_v, 25, precision=prec, dist=dist)
    per_row = (8 if prec == "fp32" else 4) // d_s  # bath vectors in one 32-byte row
    block = (1 << 13) * (-(-n_v // per_row)) * 32  # 2^13 states x padded slices x 32 bytes
    spmm2 = {"slices": [], "betas": []}
    ws = nbytes
    while ws > block:
        ctx.attach_workspace(ws)
        try:
            ctx.profile(True)
            got = ham.estimate(betas, n_v, 25, 8, precision=prec, dist=dist, full=True, passes="recompute")
            st = ctx.profile_stats()
            ctx.profile(False)
        except lib.RdmError as e:
            assert e.status == lib.ENOMEM
            break
        finally:
            ctx.detach_workspace()
        for key in ("rho", "lnZ", "gram_l"):
            np.testing.assert_array_equal(got[key], ref[key])
        sweeps, written = st["psi_init"]["launches"], st["psi_init"]["bytes"] / block
        if sweeps > 1:
            mode = "slices" if written == 1 + len(betas) else "betas"
            if mode == "betas":
                assert written == sweeps + len(betas)
            spmm2[mode].append(st["spmm_pass2"]["bytes"])
        ws -= block // 8
    assert spmm2["slices"] and spmm2["betas"]
    assert max(spmm2["slices"]) < min(spmm2["betas"])


@pytest.mark.parametrize("prec,tol,n_v,form", [("fp32", 2e-6, 16, "gram"), ("fp64", 1e-12, 16, "gram"),
                                               ("fp32", 2e-6, 14, "quadrature")])
def test_one_pass_shards_when_a_shards_basis_fits(ctx, lib, prec, tol, n_v, form):
    """passes="auto" with a caller workspace too small for the whole Krylov basis but
    large enough for that of a group of slices: the bath vectors run in consecutive
    shards that each keep their basis (one pass of the recurrence, no pass-2 launch),
    folded on the host with each shard's shift. Against the stored-basis run of all
    vectors: the same T_l and E0 (the recurrences of a slice do not depend on the others;
    the SpMM's partial sums may group differently), rho* and the per-vector Grams within
    rounding (the shards' shifts differ), and about half the SpMM bytes of the recompute
    mode in the same workspace. Also with a padded last shard (n_v = 14) and the
    quadrature form as the reported one."""
    spec = W.long_range_xxz(13, 1, 1.0, 1.0, 0.1)
    ham = lib.Hamiltonian(ctx, spec)
    betas = list(W.beta_grid(5, 0.1, 10.0))
    k = 25
    ref = ham.estimate(betas, n_v, k, 8, precision=prec, dist="gauss", form=form, full=True, passes="store")
    store_bytes = ham.workspace_size(len(betas), n_v, k, precision=prec, dist="gauss", passes="store")
    launches = {}
    for passes in ("auto", "recompute"):
        ctx.attach_workspace(int(store_bytes * 0.6))
        try:
            ctx.profile(True)
            got = ham.estimate(betas, n_v, k, 8, precision=prec, dist="gauss", form=form, full=True,
                               passes=passes)
            st = ctx.profile_stats()
            ctx.profile(False)
        finally:
            ctx.detach_workspace()
        launches[passes] = st["spmm_pass1"]["bytes"] + st.get("spmm_pass2", {"bytes": 0.0})["bytes"]
        if passes == "auto":
            assert st.get("psi_init", {"launches": 0})["launches"] == 0
            scale = np.abs(ref["t_a"]).max()
            np.testing.assert_allclose(got["t_a"], ref["t_a"], atol=tol * scale, rtol=0)
            np.testing.assert_allclose(got["t_b"], ref["t_b"], atol=tol * scale, rtol=0)
            assert abs(got["e0"] - ref["e0"]) <= tol * scale
        np.testing.assert_allclose(got["rho"], ref["rho"], atol=tol, rtol=0)
        np.testing.assert_allclose(got["lnZ"], ref["lnZ"], atol=10 * tol, rtol=0)
        np.testing.assert_allclose(got["gram_l"], ref["gram_l"], atol=tol * np.abs(ref["gram_l"]).max(), rtol=0)
    assert launches["auto"] < 0.6 * launches["recompute"]


# ---------------------------------------------------------------- bath-vector shards

@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_shards_combine_to_the_whole_run(ctx, lib, prec, tol):
    """Three shards of the bath vectors (first_vector offsets), run one after another
    on this GPU and folded on the host, equal the single run (float32: the SpMM's
    per-block reductions group the states differently with the number of slices, so
    rounding differs at ~1e-7)."""
    from paper_2204_08147_gb300.sharded import combine, local_part
    spec = W.long_range_tfim(12, 2, 1.5, 0.9)
    ham = lib.Hamiltonian(ctx, spec)
    betas = [0.5, 2.0, 7.0]
    whole = ham.estimate(betas, 10, 24, 31, precision=prec, dist="gauss")
    parts = [local_part(ham, betas, 10, 24, 31, r, 3, precision=prec, dist="gauss") for r in range(3)]
    res = combine(parts, betas, spec.d_b, 10)
    assert abs(res["e0"] - whole["e0"]) < (1e-12 if prec == "fp64" else tol) * max(1.0, abs(whole["e0"]))
    np.testing.assert_allclose(res["rho"], whole["rho"], atol=tol)
    np.testing.assert_allclose(res["lnZ"], whole["lnZ"], atol=tol)
    # and against the oracle
    ref = lanczos.Estimator(spec).run(betas, 10, 24, 31, "gauss")
    np.testing.assert_allclose(res["rho"], ref["rho"], atol=TOL64 if prec == "fp64" else TOL32)


# ---------------------------------------------------------------- bath partition, H* with its constant

@pytest.mark.parametrize("dist", ["gauss", "rademacher"])
def test_bath_hamiltonian_draws_the_same_bath_vectors(ctx, lib, dist):
    """eq. H_est takes numerator and denominator over the same v_l: the bath model's
    starting vectors equal the system-index-0 rows of the total model's block."""
    torch = _torch()
    spec = W.random_model(9, 2, 94)
    tot = lib.Hamiltonian(ctx, spec)
    bath = lib.Hamiltonian(ctx, spec, part="bath")
    assert bath.n_sites == 7 and bath.d_s == 1
    n_v, d_b = 4, 1 << 7
    xt = torch.empty((1 << 9, 4 * n_v), dtype=torch.float64, device="cuda")
    xb = torch.empty((d_b, n_v), dtype=torch.float64, device="cuda")
    tot.starting_block(xt, n_v, 77, dist)
    bath.starting_block(xb, n_v, 77, dist)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(xt.cpu().numpy()[:d_b, 0::4], xb.cpu().numpy())


def test_bath_ln_z_exhaustive_is_exact(ctx, lib):
    spec = W.random_model(9, 2, 95)
    bath = lib.Hamiltonian(ctx, spec, part="bath")
    betas = [0.2, 1.0, 3.0]
    d_b = 1 << 7
    out = bath.estimate(betas, d_b, d_b + 2, 0, precision="fp64", dist="basis")
    for i, b in enumerate(betas):
        assert abs(out["lnZ"][i] - exact.bath_log_partition(spec, b)) < 1e-9


def test_bath_ln_z_matches_oracle_same_seed(ctx, lib):
    """Lanczos quadrature for ln Z_b on the (tiled, N_b = 11) bath model against the
    oracle run on the same Gaussian vectors."""
    spec = W.random_model(12, 1, 96)
    bath = lib.Hamiltonian(ctx, spec, part="bath")
    betas = [0.5, 2.0]
    out = bath.estimate(betas, 6, 30, 5, precision="fp64", dist="gauss")
    ref = lanczos.Estimator(W.bath_spec(spec)).run(betas, 6, 30, 5, "gauss")
    np.testing.assert_allclose(out["lnZ"], ref["lnZ"], atol=1e-9, rtol=0)


def test_absolute_mean_force_and_energy_deviation_app_c(ctx, lib):
    """App. C chain, exhaustive bath vectors on both models: the eigenvalues of H*
    with its constant and the internal-energy deviation against the closed form."""
    n, j, h = 8, 1.0, 0.3
    spec = W.xy_open_chain(n, 2, j, h)
    tot = lib.Hamiltonian(ctx, spec)
    bath = lib.Hamiltonian(ctx, spec, part="bath")
    betas = [0.7, 1.3]
    d_b = 1 << (n - 2)
    rt = tot.estimate(betas, d_b, (1 << n) // 4 + 2, 0, precision="fp64", dist="basis")
    rb = bath.estimate(betas, d_b, d_b + 2, 0, precision="fp64", dist="basis")
    hs = lib.system_hamiltonian(spec)
    for i, beta in enumerate(betas):
        hstar = lib.mean_force_abs(rt["rho"][i], beta, rt["lnZ"][i], rb["lnZ"][i])
        np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(hstar)),
                                   np.sort(closed_form.mean_force_eigenvalues(n, beta, j, h)), atol=1e-9)
        p = closed_form.rho_eigenvalues(n, beta, j, h)
        want = (float(-np.sum(p * np.log(p))) - closed_form.log_z_star(n, beta, j, h)) / beta \
            - closed_form.mean_energy_chain(2, beta, j, h)
        assert abs(lib.energy_deviation(rt["rho"][i], hstar, hs, beta) - want) < 1e-9


def test_energy_deviation_lr_tfim_fp32_vs_oracle(ctx, lib):
    """float32 path end to end (rho*, ln Z_t, ln Z_b, H*, deviation) against the oracle
    estimator on the same Gaussian vectors."""
    spec = W.long_range_tfim(12, 2, 1.5, 0.8)
    betas = [1.0]
    n_v, k, seed = 16, 40, 31
    rt = lib.Hamiltonian(ctx, spec).estimate(betas, n_v, k, seed, precision="fp32", dist="gauss")
    rb = lib.Hamiltonian(ctx, spec, part="bath").estimate(betas, n_v, k, seed, precision="fp32", dist="gauss")
    ot = lanczos.Estimator(spec).run(betas, n_v, k, seed, "gauss")
    ob = lanczos.Estimator(W.bath_spec(spec)).run(betas, n_v, k, seed, "gauss")
    hs = lib.system_hamiltonian(spec)
    hstar = lib.mean_force_abs(rt["rho"][0], 1.0, rt["lnZ"][0], rb["lnZ"][0])
    href = post.mean_force(ot["rho"][0], 1.0, ot["lnZ"][0] - ob["lnZ"][0])
    np.testing.assert_allclose(hstar, href, atol=2e-3)
    dev = lib.energy_deviation(rt["rho"][0], hstar, hs, 1.0)
    dref = post.energy_deviation(ot["rho"][0], href, np.real(spin_ops.subsystem_hamiltonian(spec, "sys")), 1.0)
    assert abs(dev - dref) < 2e-3


# ---------------------------------------------------------------- c3 / c5 shapes (reduced N)

def test_c3_shape_two_pass_fp32_vs_oracle(ctx, lib):
    """The c3 configuration's structure at N = 14: all-to-all XX+YY+ZZ (alpha = 1,
    Delta = 1, h = 0.1; flip patterns with several terms and partner rows off the
    diagonal of the tile), N_s = 1, Rademacher vectors, 32 betas in [0.1, 10],
    recomputed basis, float32."""
    spec = W.long_range_xxz(14, 1, alpha=1.0, delta=1.0, h=0.1)
    betas = W.beta_grid(32, 0.1, 10.0)
    ham = lib.Hamiltonian(ctx, spec)
    out = ham.estimate(betas, 16, 40, 20220420, precision="fp32", dist="rademacher", passes="recompute")
    ref = lanczos.Estimator(spec).run(betas, 16, 40, 20220420, "rademacher")
    np.testing.assert_allclose(out["rho"], ref["rho"], atol=TOL32, rtol=0)
    np.testing.assert_allclose(out["lnZ"], ref["lnZ"], rtol=1e-5, atol=1e-4)


def test_c5_shape_two_pass_fp32_vs_oracle(ctx, lib):
    """The c5 configuration's structure at N = 15: alpha = 1.5, Delta = 0.5, N_s = 1,
    n_v = 4 Rademacher (one 8-column slice), k = 50, beta = 2, recomputed basis."""
    spec = W.long_range_xxz(15, 1, alpha=1.5, delta=0.5)
    ham = lib.Hamiltonian(ctx, spec)
    out = ham.estimate([2.0], 4, 50, 20220421, precision="fp32", dist="rademacher", passes="recompute")
    ref = lanczos.Estimator(spec).run([2.0], 4, 50, 20220421, "rademacher")
    np.testing.assert_allclose(out["rho"], ref["rho"], atol=TOL32, rtol=0)
    np.testing.assert_allclose(out["lnZ"], ref["lnZ"], rtol=1e-5, atol=1e-4)


# ---------------------------------------------------------------- per-column (block size 1) recurrences

@pytest.mark.parametrize("passes", ["store", "recompute"])
def test_single_recurrence_matches_oracle_fp64(ctx, lib, passes):
    """recurrence="single": one Lanczos recurrence per column e_i (x) v_l (Sec. 4.2), Gram
    cross terms psi_i^T psi_j, against the oracle's per-column run on the same vectors."""
    spec = W.random_model(10, 1, 31)
    betas = [0.5, 2.0]
    ham = lib.Hamiltonian(ctx, spec)
    out = ham.estimate(betas, 5, 20, 8, precision="fp64", dist="gauss", full=True, passes=passes,
                       recurrence="single")
    ref = lanczos.Estimator(spec).run(betas, 5, 20, 8, "gauss", block=False)
    np.testing.assert_allclose(out["rho"], ref["rho"], atol=TOL64, rtol=0)
    np.testing.assert_allclose(out["lnZ"], ref["lnZ"], atol=1e-9, rtol=0)
    np.testing.assert_allclose(out["gram_l"], ref["gram_l"], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(out["quad_l"], ref["quad_l"], rtol=1e-9, atol=1e-12)
    assert abs(out["e0"] - ref["e0"]) < 1e-10


def test_single_recurrence_store_and_recompute_bit_identical(ctx, lib):
    spec = W.long_range_tfim(12, 2, 1.5, 0.6)
    ham = lib.Hamiltonian(ctx, spec)
    a = ham.estimate([0.5, 1.5], 8, 25, 3, precision="fp32", dist="gauss", full=True, passes="store",
                     recurrence="single")
    b = ham.estimate([0.5, 1.5], 8, 25, 3, precision="fp32", dist="gauss", full=True, passes="recompute",
                     recurrence="single")
    for key in ("rho", "lnZ", "gram_l", "quad_l", "t_a", "t_b"):
        np.testing.assert_array_equal(a[key], b[key])


def test_single_recurrence_fp32_tiled_vs_oracle(ctx, lib):
    """d_s = 4 on the tiled SpMM with block size 1: 32 columns of 8 bath vectors."""
    spec = W.long_range_tfim(12, 2, 1.5, 1.1)
    ham = lib.Hamiltonian(ctx, spec)
    out = ham.estimate([1.0], 8, 30, 20220418, precision="fp32", dist="gauss", recurrence="single")
    ref = lanczos.Estimator(spec).run([1.0], 8, 30, 20220418, "gauss", block=False)
    np.testing.assert_allclose(out["rho"], ref["rho"], atol=TOL32)
    assert abs(out["lnZ"][0] - ref["lnZ"][0]) < 1e-3


def test_single_recurrence_exhaustive_is_exact(ctx, lib):
    spec = W.random_model(7, 1, 32)
    betas = [0.3, 2.5]
    ham = lib.Hamiltonian(ctx, spec)
    out = ham.estimate(betas, spec.d_b, spec.dim + 2, 0, precision="fp64", dist="basis", recurrence="single")
    rho, lnz = exact.exact_rho(spec, betas)
    np.testing.assert_allclose(out["rho"], rho, atol=TOL64, rtol=0)
    np.testing.assert_allclose(out["lnZ"], lnz, atol=1e-9, rtol=0)


def test_single_recurrence_rejects_fp64_with_four_system_states(ctx, lib):
    ham = lib.Hamiltonian(ctx, W.random_model(8, 2, 33))
    with pytest.raises(lib.RdmError) as e:
        ham.estimate([1.0], 2, 5, 1, precision="fp64", recurrence="single")
    assert e.value.status == lib.EINVAL


def test_block_recurrence_more_accurate_than_single(ctx, lib):
    """Sec. 4.2's remark on the GPU path: at equal k the block recurrence is closer to
    the exact-function estimator (same vectors) than per-column recurrences."""
    spec = W.random_model(10, 2, 5)
    h = spin_ops.dense_hamiltonian(spec)
    rho2, _ = lanczos.exact_function_estimator(spec, h, [2.0], 6, 3, "gauss")
    ham = lib.Hamiltonian(ctx, spec)
    for k in (4, 6, 8):
        b = ham.estimate([2.0], 6, k, 3, precision="fp32", dist="gauss")
        s = ham.estimate([2.0], 6, k, 3, precision="fp32", dist="gauss", recurrence="single")
        assert np.abs(b["rho"] - rho2).max() < np.abs(s["rho"] - rho2).max()


# ---------------------------------------------------------------- bath order (ladder)

@pytest.mark.parametrize("prec,tol", [("fp64", TOL64), ("fp32", TOL32)])
def test_reordered_bath_bits_match_oracle(lib, prec, tol):
    """The ladder of Sec. 5.2 numbered leg by leg (14 spins, system = rung 2): the
    library stores it with its bath bits reordered (fewer partner tiles), draws the bath
    vectors in the caller's order, and matches the oracle run on the caller's numbering;
    with the reordering switched off the result agrees to rounding."""
    spec = W.spin_ladder(7, 2, numbering="leg")
    order, before, after = lib.bath_order(spec)
    assert after < before and order != list(range(14))
    betas = [0.5, 2.0]
    ctx = lib.Context(0)
    try:
        ham = lib.Hamiltonian(ctx, spec)
        out = ham.estimate(betas, 6, 24, 77, precision=prec, dist="gauss", full=True)
        ctx.set_bath_order(False)
        plain = lib.Hamiltonian(ctx, spec).estimate(betas, 6, 24, 77, precision=prec, dist="gauss", full=True)
    finally:
        ctx.close()
    ref = lanczos.Estimator(spec).run(betas, 6, 24, 77, "gauss")
    np.testing.assert_allclose(out["rho"], ref["rho"], atol=tol, rtol=0)
    np.testing.assert_allclose(out["rho"], plain["rho"], atol=1e-13 if prec == "fp64" else 1e-5, rtol=0)
    np.testing.assert_allclose(out["t_a"][:, :6], plain["t_a"][:, :6], atol=1e-12 if prec == "fp64" else 1e-4)


def test_reordered_ham_keeps_caller_order_for_apply_and_starting_block(lib):
    """rdm_apply_hamiltonian and rdm_starting_block of a reordered Hamiltonian act in the
    caller's state order: bit-exact against the oracle's tensor-leg H on an
    integer-valued ladder, and the starting block against the generator."""
    import torch
    spec = W.spin_ladder(7, 2, j_leg=2.0, j_rung=-1.0, h=2.0, numbering="leg")
    assert lib.bath_order(spec)[0] != list(range(14))
    ctx = lib.Context(0)
    try:
        ham = lib.Hamiltonian(ctx, spec)
        rng = np.random.default_rng(3)
        x = rng.integers(-3, 4, size=(1 << 14, 4)).astype(np.float64)
        xd = torch.tensor(x, device="cuda")
        yd = torch.empty_like(xd)
        ham.apply(xd, yd)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(yd.cpu().numpy(), spin_ops.TensorHamiltonian(spec)(x))
        blk = torch.empty((1 << 14, 4 * 2), dtype=torch.float64, device="cuda")
        ham.starting_block(blk, 2, 11, "rademacher")
        torch.cuda.synchronize()
        want = np.hstack([orng.starting_block(4, orng.bath_vector(1 << 12, l, 11, "rademacher")) for l in range(2)])
        np.testing.assert_array_equal(blk.cpu().numpy(), want)
    finally:
        ctx.close()


# ---------------------------------------------------------------- small dense step on the device

@pytest.mark.parametrize("spec_fn,n_v,k,betas,dist", [
    (lambda: W.long_range_tfim(12, 2, 1.5, 1.1), 6, 40, list(W.beta_grid(20, 0.05, 10.0)) + [0.0], "gauss"),
    (lambda: W.long_range_xxz(11, 1, 1.0, 1.0, 0.1), 5, 60, [0.3, 3.0, 12.0], "rademacher"),
    (lambda: W.random_model(9, 2, 31), 3, 25, [1.0, 4.0], "gauss"),
    (lambda: W.xxz_chain(10, 1, 1.0, 0.5), 16, 40, [0.5, 1.0, 2.0], "rademacher"),
])
def test_device_dense_step_matches_host_and_oracle(lib, spec_fn, n_v, k, betas, dist):
    """The device small dense step (multisection for lambda_min, Chebyshev expansion of
    exp(-beta (T - E0)/2) E1) against the host eigendecomposition on the same T (float64
    path: per-vector Gram and quadrature forms within 1e-12 of their trace, E0 within
    1e-12 |E0|), and the estimate against the oracle at the float64 tolerance. Covers
    more than one chunk of 16 betas, beta = 0 and beta up to 12."""
    spec = spec_fn()
    ctx = lib.Context(0)
    try:
        ham = lib.Hamiltonian(ctx, spec)
        ctx.set_device_dense(2)
        dev = ham.estimate(betas, n_v, k, 9, precision="fp64", dist=dist, full=True)
        ctx.set_device_dense(0)
        host = ham.estimate(betas, n_v, k, 9, precision="fp64", dist=dist, full=True)
    finally:
        ctx.close()
    assert abs(dev["e0"] - host["e0"]) <= 1e-12 * max(1.0, abs(host["e0"]))
    for key in ("gram_l", "quad_l"):
        tr = np.trace(host[key], axis1=2, axis2=3)[..., None, None]
        assert np.abs(dev[key] - host[key]).max() <= 1e-12 * tr.max()
        assert np.all(np.abs(dev[key] - host[key]) <= 1e-12 * tr)
    ref = lanczos.Estimator(spec).run(betas, n_v, k, 9, dist)
    np.testing.assert_allclose(dev["rho"], ref["rho"], atol=TOL64, rtol=0)


def test_device_dense_step_is_used_and_large_t_falls_back(lib):
    """By default the device step (dense_fT in the profile) runs for grids of 8 or more
    betas and the host path for fewer; a T too large for the device step's shared memory
    (k d_s^2 > 5120) takes the host path and still matches the oracle."""
    spec = W.random_model(8, 2, 5)
    ctx = lib.Context(0)
    try:
        ham = lib.Hamiltonian(ctx, spec)
        ctx.profile(True)
        ham.estimate([1.0, 2.0], 2, 20, 3, precision="fp64", dist="gauss")  # 2 betas: host
        ham.estimate(W.beta_grid(8, 0.5, 4.0), 2, 20, 3, precision="fp64", dist="gauss")  # 8: device
        st = ctx.profile_stats()
        ctx.profile(False)
        assert st["dense_fT"]["launches"] == 1
        big = ham.estimate(W.beta_grid(8, 0.5, 4.0), 1, 330, 3, precision="fp64", dist="gauss")  # 5280
        ref = lanczos.Estimator(spec).run(W.beta_grid(8, 0.5, 4.0), 1, 330, 3, "gauss")
        np.testing.assert_allclose(big["rho"], ref["rho"], atol=1e-8, rtol=0)
    finally:
        ctx.close()


@pytest.mark.parametrize("n,n_sys,fields", [(13, 1, 0), (14, 0, 0), (15, 2, 0), (14, 1, 2), (16, 2, 5)])
@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_apply_tiled_bit_exact_hopping_pairs(ctx, lib, n, n_sys, fields, dtype):
    """All-to-all XX + YY with J^x = J^y (the long-range XXZ shape: every pair hops only
    antiparallel spins, a coefficient that depends on the parity of the flipped pair) on
    integer couplings: the tiled SpMM's parity-only paths -- one load per pair of
    register rows, partner tiles of single high pairs with a tile-uniform coefficient,
    and the partner tiles of one high spin consumed in opposite-spin pairs (with an
    uneven split of down and up spins on most tiles) -- equal H x bit for bit. With
    `fields` transverse fields on the first sites (the high spins of the tile), those
    spins' partner groups also carry a single flip and are not paired."""
    torch = _torch()
    rng = np.random.default_rng(n)
    spec = W.long_range_xxz(n, n_sys, 0.0, 1.0, 0.0)
    c = rng.integers(1, 4, size=(n, n)).astype(np.float64)
    spec.jx[:] = np.triu(c, 1)
    spec.jy[:] = spec.jx
    spec.jz[:] = np.triu(rng.integers(-2, 3, size=(n, n)).astype(np.float64), 1)
    spec.hz[:] = rng.integers(-2, 3, size=n)
    spec.gx[:fields] = rng.integers(1, 3, size=fields)
    h = spin_ops.sparse_hamiltonian(spec)
    ncols = 8 if dtype == "float32" else 4
    x = rng.integers(-3, 4, size=(1 << n, ncols)).astype(np.float64)
    ham = lib.Hamiltonian(ctx, spec)
    xd = torch.from_numpy(x).to(getattr(torch, dtype)).cuda()
    yd = torch.empty_like(xd)
    ham.apply(xd, yd)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(yd.double().cpu().numpy(), h @ x)


def test_spmm_forms_agree_and_the_default_follows_the_tile_count(lib):
    """The estimator with the tiled SpMM (form 1), the plain one (form 2) and the default
    (form 0): the same estimate within float64 rounding; the default is the plain kernel
    for a block of 8 tiles (the c1 chain, one tile per slice) and the tiled one for 512
    tiles (N = 16, 8 slices), bit for bit."""
    ctx = lib.Context(0)
    try:
        for spec, n_v, tiled in ((W.config_c1()["spec"], 16, False), (W.long_range_xxz(16, 1, 1.0, 1.0, 0.1), 16, True)):
            ham = lib.Hamiltonian(ctx, spec)
            outs = {}
            for form in (0, 1, 2):
                ctx.set_spmm_form(form)
                outs[form] = ham.estimate([0.5, 1.0], n_v, 30, 7, precision="fp64", dist="rademacher", full=True)
            np.testing.assert_allclose(outs[1]["rho"], outs[2]["rho"], atol=1e-13, rtol=0)
            same = outs[1] if tiled else outs[2]
            for key in ("rho", "gram_l", "t_a", "t_b"):
                np.testing.assert_array_equal(outs[0][key], same[key])
            ham.close()
        with pytest.raises(lib.RdmError) as e:
            ctx.set_spmm_form(3)
        assert e.value.status == lib.EINVAL
    finally:
        ctx.close()
