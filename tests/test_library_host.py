"""Host-side checks of the C-ABI library (no GPU needed): symbols, host math, errors."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rdm():
    from paper_2204_08147_gb300 import build
    if not os.path.exists(build.LIB):
        build.build_library()
    from paper_2204_08147_gb300 import rdm as mod
    return mod


def _declared_functions():
    txt = open(os.path.join(ROOT, "include", "rdm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rdm_[a-z_]+)\s*\(", txt)))


def test_library_exports_every_declared_function(rdm):
    names = _declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(rdm._lib, n), f"{n} declared in include/rdm.h but not exported"


def test_symmetric_eig_matches_numpy(rdm):
    rng = np.random.default_rng(0)
    for n in (1, 2, 3, 7, 40, 121):
        a = rng.normal(size=(n, n))
        a = a + a.T
        w, v = rdm.symmetric_eig(a)
        np.testing.assert_allclose(w, np.linalg.eigvalsh(a), atol=1e-12 * max(1, np.abs(a).max()) * n)
        np.testing.assert_allclose(v.T @ v, np.eye(n), atol=1e-12 * n)
        np.testing.assert_allclose(a @ v, v * w, atol=1e-11 * n)


def test_symmetric_eig_block_tridiagonal_and_degenerate(rdm):
    rng = np.random.default_rng(1)
    p, k = 4, 30
    t = np.zeros((p * k, p * k))
    for j in range(k):
        a = rng.normal(size=(p, p))
        t[j * p:(j + 1) * p, j * p:(j + 1) * p] = a + a.T
        if j + 1 < k:
            b = np.triu(rng.normal(size=(p, p)))
            t[(j + 1) * p:(j + 2) * p, j * p:(j + 1) * p] = b
            t[j * p:(j + 1) * p, (j + 1) * p:(j + 2) * p] = b.T
    w, v = rdm.symmetric_eig(t)
    np.testing.assert_allclose(w, np.linalg.eigvalsh(t), atol=1e-11)
    np.testing.assert_allclose(t @ v, v * w, atol=1e-10)
    # exactly degenerate spectrum and a decoupled zero block
    d = np.diag([2.0, 2.0, 2.0, -1.0, 0.0, 0.0])
    q, _ = np.linalg.qr(rng.normal(size=(6, 6)))
    m = q @ d @ q.T
    w, v = rdm.symmetric_eig(m)
    np.testing.assert_allclose(w, [-1, 0, 0, 2, 2, 2], atol=1e-13)
    np.testing.assert_allclose(v.T @ v, np.eye(6), atol=1e-13)


def _block_tridiagonal(rng, p, k, scale=1.0):
    t = np.zeros((p * k, p * k))
    for j in range(k):
        a = rng.normal(size=(p, p)) * scale
        t[j * p:(j + 1) * p, j * p:(j + 1) * p] = a + a.T
        if j + 1 < k:
            b = np.triu(rng.normal(size=(p, p))) * scale
            t[(j + 1) * p:(j + 2) * p, j * p:(j + 1) * p] = b
            t[j * p:(j + 1) * p, (j + 1) * p:(j + 2) * p] = b.T
    return t


@pytest.mark.parametrize("p,k", [(1, 40), (2, 30), (4, 25), (4, 60), (3, 7)])
def test_function_of_t_matches_oracle(rdm, p, k):
    """The small dense step (eq. fT) on block tridiagonal T (band reduction path) and on
    a dense symmetric T (Householder path) against the oracle's eigendecomposition form."""
    from oracle import lanczos
    rng = np.random.default_rng(100 + p * k)
    betas = [0.0, 0.3, 1.0, 4.0]
    for t in (_block_tridiagonal(rng, p, k), None):
        if t is None:
            x = rng.normal(size=(p * k, p * k))
            t = x + x.T
        tmin, c = rdm.function_of_t(t, p, betas)
        w = np.linalg.eigvalsh(t)
        assert abs(tmin - w[0]) < 1e-12 * max(1.0, np.abs(w).max())
        for bi, beta in enumerate(betas):
            ref = lanczos.function_of_t_first_block(t, p, lambda x: np.exp(-beta * (x - tmin) / 2.0))
            np.testing.assert_allclose(c[bi], ref, atol=1e-12 * np.sqrt(p * k), rtol=0)


def test_function_of_t_degenerate_and_errors(rdm):
    """Exactly degenerate spectra and decoupled blocks (a Krylov breakdown leaves B_j = 0),
    and the argument checks."""
    rng = np.random.default_rng(7)
    q, _ = np.linalg.qr(rng.normal(size=(8, 8)))
    t = q @ np.diag([1.0, 1.0, 1.0, -2.0, 0.5, 0.5, 3.0, 3.0]) @ q.T
    tmin, c = rdm.function_of_t(t, 2, [1.5])
    assert abs(tmin + 2.0) < 1e-13
    w, v = np.linalg.eigh(t)
    ref = (v * np.exp(-1.5 * (w - tmin) / 2)) @ v[:2, :].T
    np.testing.assert_allclose(c[0], ref, atol=1e-13)
    blk = _block_tridiagonal(rng, 2, 10)
    blk[8:10, 6:8] = blk[6:8, 8:10] = 0.0  # B_4 = 0: T splits
    tmin, c = rdm.function_of_t(blk, 2, [2.0])
    w, v = np.linalg.eigh(blk)
    np.testing.assert_allclose(c[0], (v * np.exp(-(w - tmin))) @ v[:2, :].T, atol=1e-12)
    np.testing.assert_allclose(c[0][8:], 0.0, atol=1e-14)  # E1 never reaches the lower part
    for bad in [(np.eye(3), 4, [1.0]), (np.eye(3), 1, [-1.0]), (np.eye(3), 1, [float("inf")]),
                (np.full((3, 3), np.nan), 1, [1.0])]:
        with pytest.raises(rdm.RdmError) as e:
            rdm.function_of_t(*bad)
        assert e.value.status == rdm.EINVAL


def test_function_of_t_batch_on_the_worker_pool(rdm):
    """The batched small dense step (the host worker pool) equals the one-matrix call
    bit for bit, also with several callers running jobs on the pool at once."""
    import threading
    rng = np.random.default_rng(11)
    ts = np.stack([_block_tridiagonal(rng, 4, 20) for _ in range(13)])
    betas = [0.5, 2.0]
    ref = [rdm.function_of_t(t, 4, betas) for t in ts]
    tmin, c = rdm.function_of_t_batch(ts, 4, betas)
    for r, (tm, cr) in enumerate(ref):
        assert tmin[r] == tm
        np.testing.assert_array_equal(c[r], cr)
    outs, errs = [None] * 6, []

    def worker(i):
        try:
            outs[i] = rdm.function_of_t_batch(ts[i:i + 8], 4, betas)
        except Exception as e:  # noqa: BLE001
            errs.append(e)
    th = [threading.Thread(target=worker, args=(i,)) for i in range(6)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errs
    for i, (tm, cc) in enumerate(outs):
        np.testing.assert_array_equal(tm, tmin[i:i + 8])
        np.testing.assert_array_equal(cc, c[i:i + 8])
    with pytest.raises(rdm.RdmError) as e:
        rdm.function_of_t_batch(np.full((2, 3, 3), np.nan), 1, [1.0])
    assert e.value.status == rdm.EINVAL


def test_mean_force_and_entropy_match_oracle(rdm):
    from oracle import post
    rng = np.random.default_rng(2)
    for d in (1, 2, 4, 8):
        x = rng.normal(size=(d, d))
        rho = x @ x.T + 0.1 * np.eye(d)
        rho /= np.trace(rho)
        beta = 0.7
        np.testing.assert_allclose(rdm.mean_force(rho, beta), post.mean_force(rho, beta), atol=1e-12)
        assert abs(rdm.entropy(rho) - post.entropy(rho)) < 1e-13
    assert abs(rdm.entropy(np.eye(4) / 4) - np.log(4)) < 1e-14
    assert abs(rdm.entropy(np.diag([1.0, 0.0]))) == 0.0


def test_absolute_mean_force_and_energy_deviation_match_oracle(rdm):
    from oracle import post
    rng = np.random.default_rng(3)
    for d in (1, 2, 4):
        x = rng.normal(size=(d, d))
        rho = x @ x.T + 0.1 * np.eye(d)
        rho /= np.trace(rho)
        y = rng.normal(size=(d, d))
        hs = y + y.T
        beta, ln_zt, ln_zb = 0.7, 3.1, 2.4
        hstar = rdm.mean_force_abs(rho, beta, ln_zt, ln_zb)
        np.testing.assert_allclose(hstar, post.mean_force(rho, beta, ln_zt - ln_zb), atol=1e-12)
        assert abs(rdm.energy_deviation(rho, hstar, hs, beta) - post.energy_deviation(rho, hstar, hs, beta)) < 1e-12
    with pytest.raises(rdm.RdmError) as e:
        rdm.mean_force_abs(np.eye(2) / 2, 1.0, float("nan"), 0.0)
    assert e.value.status == rdm.EINVAL


@pytest.mark.parametrize("n,n_sys,seed", [(5, 1, 90), (6, 2, 91), (4, 2, 92), (3, 0, 93)])
def test_system_hamiltonian_matches_oracle(rdm, n, n_sys, seed):
    """H_s in the SpMM's term convention against the oracle's Kronecker-product H_s."""
    import workloads as W
    from oracle import spin_ops
    spec = W.random_model(n, n_sys, seed)
    got = rdm.system_hamiltonian(spec)
    if n_sys == 0:
        np.testing.assert_array_equal(got, np.zeros((1, 1)))
        return
    want = spin_ops.subsystem_hamiltonian(spec, "sys")
    assert np.abs(np.imag(want)).max() == 0.0
    np.testing.assert_allclose(got, np.real(want), atol=1e-13)


def test_mean_force_rejects_non_positive(rdm):
    with pytest.raises(rdm.RdmError) as e:
        rdm.mean_force(np.diag([1.0, 0.0]), 1.0)
    assert e.value.status == rdm.ENOTPD
    with pytest.raises(rdm.RdmError) as e:
        rdm.mean_force(np.eye(2) / 2, 0.0)
    assert e.value.status == rdm.EINVAL


def test_create_without_gpu_fails_cleanly(rdm):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import ctypes as C
    h = C.c_void_p()
    st = rdm._lib.rdm_create(C.byref(h), 0, None)
    assert st in (rdm.ECUDA, rdm.EINVAL)
    assert rdm.last_error()


def test_header_enums_match_binding(rdm):
    txt = open(os.path.join(ROOT, "include", "rdm.h")).read()
    for name, val in [("RDM_EINVAL", rdm.EINVAL), ("RDM_ENOMEM", rdm.ENOMEM), ("RDM_ECUDA", rdm.ECUDA),
                      ("RDM_ENOTPD", rdm.ENOTPD), ("RDM_EBUSY", rdm.EBUSY)]:
        assert re.search(rf"{name}\s*=\s*{val}\b", txt), name
    assert re.search(r"RDM_FP64\s*=\s*0", txt) and re.search(r"RDM_FP32\s*=\s*1", txt)
    assert "RDM_RADEMACHER = 0, RDM_GAUSS = 1, RDM_BASIS = 2" in txt


def test_bath_order_from_the_coupling_graph(rdm):
    """The ladder of Sec. 5.2 (10 rungs, system = one rung) numbered leg by leg: the
    library's bath order copies fewer partner tiles per tile than the caller's (13.5
    there, 8.5 for the rung-by-rung numbering, which it keeps: 5 rung and 8 leg bonds
    among the sites above the tile bits at 1/2 each -- only the antiparallel half of the
    tiles hops such a pair -- plus the two legs that leave the tile's rungs). The order
    is a permutation of the bath sites that leaves the system sites in place, and
    repeated calls give the same order."""
    import workloads as W
    for sr in (0, 2, 4):
        order, before, after = rdm.bath_order(W.spin_ladder(10, sr))
        assert before == after == 8.5 and order == list(range(20))
        spec = W.spin_ladder(10, sr, numbering="leg")
        order, before, after = rdm.bath_order(spec)
        assert before > 12.0 and after <= 9.0
        assert order[:2] == [0, 1] and sorted(order) == list(range(20))
        assert rdm.bath_order(spec) == (order, before, after)


def test_bath_order_keeps_a_model_with_no_gain(rdm):
    """Single-site flips (the transverse-field model) give one partner tile per high bit
    in any order: the caller's order is kept; below 11 sites there is nothing to move."""
    import workloads as W
    spec = W.config_c2(0)["spec"]
    order, before, after = rdm.bath_order(spec)
    assert order == list(range(22)) and before == after == 12.0
    order, before, after = rdm.bath_order(W.xxz_chain(10, 1))
    assert order == list(range(10)) and before == after == 0.0


def test_bath_order_search_skipped_for_permutation_symmetric_couplings(rdm):
    """All-to-all couplings (the long-range XXZ models, where every pair of sites hops) and
    single-site flips map onto themselves under any permutation of the bath bits, so every
    order has the same partner count and the search is skipped: the call returns at once.
    A chain is not symmetric and is searched."""
    import time
    import workloads as W
    for spec in (W.config_c2(0)["spec"], W.config_c3()["spec"], W.config_c5()["spec"]):
        t = time.perf_counter()
        order, before, after = rdm.bath_order(spec)
        assert time.perf_counter() - t < 0.02
        assert order == list(range(spec.n_sites)) and before == after > 0.0
    order, before, after = rdm.bath_order(W.xxz_chain(20, 1))
    assert sorted(order) == list(range(20)) and after <= before


def test_bath_order_reused_for_a_repeated_structure(rdm):
    """The order search depends only on the bath size and the set of (flip mask,
    parity-only) pairs: a model with the same structure and other couplings (a serving
    stream's chains or ladders) takes the order found before, at once."""
    import time
    import workloads as W
    first = rdm.bath_order(W.spin_ladder(9, 2, numbering="leg"))
    t = time.perf_counter()
    again = rdm.bath_order(W.spin_ladder(9, 2, j_leg=0.6, j_rung=1.3, numbering="leg"))
    assert time.perf_counter() - t < 0.02
    assert again == first and first[2] < first[1]


def test_context_knobs_reject_a_null_context(rdm):
    """The launch-form and mode setters validate their context before touching it."""
    for name in ("rdm_set_spmm_form", "rdm_set_packed_form", "rdm_set_device_dense", "rdm_set_bath_order",
                 "rdm_set_graphs"):
        st = getattr(rdm._lib, name)(None, 0)
        assert st == rdm.EINVAL, name
