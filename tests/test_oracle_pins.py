"""Pins of the CPU oracle against facts other than itself (no GPU needed).

Each test ties an oracle function to a closed form, a textbook spectrum, a
brute-force construction, a symmetry or limit of the paper, or an exactness
property of the algorithm, so that a dropped term, a wrong sign, a wrong index or
a transposed operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import closed_form, exact, lanczos, post, rng, spin_ops


# ---------------------------------------------------------------- Hamiltonian

def test_two_site_heisenberg_spectrum():
    # J (XX + YY + ZZ) on two spins: triplet at +J, singlet at -3J (textbook).
    jval = 0.7
    spec = W.xxz_chain(2, 1, j=jval, delta=1.0, h=0.0, periodic=False)
    ev = np.linalg.eigvalsh(spin_ops.dense_hamiltonian(spec))
    np.testing.assert_allclose(ev, [-3 * jval, jval, jval, jval], atol=1e-14)


def test_two_site_xy_anisotropic_spectrum():
    # Jx XX + Jy YY: eigenvalues +-(Jx+Jy) on the anti-aligned pair, +-(Jx-Jy) on the aligned one.
    spec = W.random_model(2, 1, seed=0, lam=1.0)
    spec.jx[0, 1], spec.jy[0, 1], spec.jz[0, 1] = 0.9, 0.4, 0.0
    spec.hz[:] = 0
    spec.gx[:] = 0
    ev = np.linalg.eigvalsh(spin_ops.dense_hamiltonian(spec))
    np.testing.assert_allclose(ev, sorted([1.3, -1.3, 0.5, -0.5]), atol=1e-14)


def _brute_force_matrix(spec):
    """<s'|H|s> from spin rules: site q is digit q of s written with N binary
    digits, most significant first; digit 0 is spin up (Z = +1)."""
    n = spec.n_sites
    d = 1 << n
    h = np.zeros((d, d))

    def digit(s, q):
        return (s >> (n - 1 - q)) & 1

    for s in range(d):
        zs = [1 - 2 * digit(s, q) for q in range(n)]
        for a in range(n):
            for b in range(a + 1, n):
                sb = (a < spec.n_sys) != (b < spec.n_sys)
                lam = spec.lambda_sb if sb else 1.0
                t = s ^ (1 << (n - 1 - a)) ^ (1 << (n - 1 - b))
                # X_a X_b flips both spins with amplitude 1.
                h[t, s] += lam * spec.jx[a, b]
                # Y|up> = i|down>, Y|down> = -i|up>: Y_a Y_b amplitude = (i z_a)(i z_b) = -z_a z_b.
                h[t, s] += lam * spec.jy[a, b] * (-zs[a] * zs[b])
                h[s, s] += lam * spec.jz[a, b] * zs[a] * zs[b]
        for q in range(n):
            h[s, s] += spec.hz[q] * zs[q]
            h[s ^ (1 << (n - 1 - q)), s] += spec.gx[q]
    return h


@pytest.mark.parametrize("n,n_sys,seed", [(3, 1, 1), (4, 2, 2), (5, 1, 3), (6, 2, 4)])
def test_dense_hamiltonian_matches_brute_force(n, n_sys, seed):
    spec = W.random_model(n, n_sys, seed)
    np.testing.assert_allclose(spin_ops.dense_hamiltonian(spec), _brute_force_matrix(spec), atol=1e-13)


@pytest.mark.parametrize("n,n_sys,seed", [(4, 1, 5), (7, 2, 6), (8, 0, 7)])
def test_tensor_apply_matches_dense(n, n_sys, seed):
    spec = W.random_model(n, n_sys, seed)
    h = spin_ops.dense_hamiltonian(spec)
    x = np.random.default_rng(seed).normal(size=(1 << n, 3))
    np.testing.assert_allclose(spin_ops.TensorHamiltonian(spec)(x), h @ x, atol=1e-12)


def test_parts_sum_to_total_and_sb_has_no_partial_trace():
    spec = W.random_model(6, 2, 8)
    tot = spin_ops.dense_hamiltonian(spec)
    hs = spin_ops.dense_hamiltonian(spec, "sys")
    hb = spin_ops.dense_hamiltonian(spec, "bath")
    hsb = spin_ops.dense_hamiltonian(spec, "sb")
    np.testing.assert_allclose(hs + hb + hsb, tot, atol=1e-13)
    # App. A: tr_b(H_sb) = 0 because every Pauli matrix is traceless.
    np.testing.assert_allclose(exact.partial_trace_bath(hsb, spec.d_s, spec.d_b), 0.0, atol=1e-12)
    # bar H_s = H_s (x) I_b (eq. 1).
    np.testing.assert_allclose(hs, np.kron(spin_ops.subsystem_hamiltonian(spec, "sys"),
                                           np.eye(spec.d_b)), atol=1e-13)


def test_norm_bound_is_a_bound():
    spec = W.random_model(7, 1, 9)
    ev = np.linalg.eigvalsh(spin_ops.dense_hamiltonian(spec))
    assert max(abs(ev[0]), abs(ev[-1])) <= spin_ops.TensorHamiltonian(spec).norm_bound() + 1e-12


# ---------------------------------------------------------------- O1 exact

@pytest.mark.parametrize("n", [6, 8, 10])
@pytest.mark.parametrize("beta", [0.2, 1.0, 3.5])
def test_exact_matches_app_c_closed_form(n, beta):
    spec = W.xy_open_chain(n, 2, j=1.0, h=0.3)
    solver = exact.ExactSolver(spec)
    rho, lnz = solver.reduced(beta)
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(rho)),
                               closed_form.rho_eigenvalues(n, beta, 1.0, 0.3), atol=1e-13)
    assert abs(lnz - closed_form.log_partition_chain(n, beta, 1.0, 0.3)) < 1e-12
    ln_zb = exact.bath_log_partition(spec, beta)
    assert abs((lnz - ln_zb) - closed_form.log_z_star(n, beta, 1.0, 0.3)) < 1e-12


def test_golden_app_c_file_matches_closed_form():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "app_c_xy_chain.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) > 10
    for r in rows:
        n, beta = int(r[0]), float(r[1])
        p = np.array([float(x) for x in r[2:6]])
        np.testing.assert_allclose(p, closed_form.rho_eigenvalues(n, beta, 1.0, 0.3), rtol=0, atol=1e-15)
        assert abs(float(r[6]) - closed_form.log_z_star(n, beta, 1.0, 0.3)) < 1e-12


def test_high_temperature_limit():
    spec = W.random_model(6, 2, 11)
    rho, _ = exact.exact_rho(spec, [0.0])
    np.testing.assert_allclose(rho[0], np.eye(4) / 4, atol=1e-15)
    # Sec. 2.3: H*(beta) = H_s + O(beta) since tr_b H_sb = 0; compare traceless parts.
    beta = 1e-4
    rho, _ = exact.exact_rho(spec, [beta])
    hstar = post.mean_force(rho[0], beta)
    hs = spin_ops.subsystem_hamiltonian(spec, "sys")
    dev = (hstar - np.trace(hstar) / 4 * np.eye(4)) - (hs - np.trace(hs) / 4 * np.eye(4))
    assert np.abs(dev).max() < 50 * beta


def test_uncoupled_limit_gives_bare_system_gibbs():
    spec = W.random_model(7, 2, 12, lam=0.0)
    for beta in [0.4, 2.0]:
        rho, _ = exact.exact_rho(spec, [beta])
        np.testing.assert_allclose(rho[0], exact.bare_system_gibbs(spec, beta), atol=1e-13)


def test_low_temperature_limit_is_ground_state_reduced():
    spec = W.random_model(6, 1, 13)
    solver = exact.ExactSolver(spec)
    gap = solver.evals[1] - solver.evals[0]
    assert gap > 1e-3
    beta = 40.0 / gap
    rho, _ = solver.reduced(beta)
    np.testing.assert_allclose(rho, solver.ground_state_reduced(), atol=1e-10)


def test_c1_symmetry_gives_maximally_mixed():
    # h = 0 XXZ chain: spin-flip and U(1) symmetry force rho* = I/2, S = ln 2.
    c = W.config_c1()
    rho, _ = exact.exact_rho(c["spec"], c["betas"])
    for r in rho:
        np.testing.assert_allclose(r, np.eye(2) / 2, atol=1e-14)
        assert abs(post.entropy(r) - math.log(2)) < 1e-13


# ---------------------------------------------------------------- RNG

def test_rng_scalar_and_vector_forms_agree():
    ctr = np.array([1, 2, 3, (5 << 40) | 7, (1 << 63) + 11], dtype=np.uint64)
    vec = rng.splitmix64_array(12345, ctr)
    for c, v in zip(ctr, vec):
        assert int(v) == rng.splitmix64(12345, int(c))


def test_rademacher_vectors():
    d_b = 1 << 12
    v = rng.bath_vector(d_b, 3, 99, "rademacher")
    assert set(np.unique(v * math.sqrt(d_b))) == {-1.0, 1.0}
    assert abs(v @ v - 1.0) < 1e-14
    assert abs(np.mean(np.sign(v))) < 5 / math.sqrt(d_b)  # balanced signs
    w = rng.bath_vector(d_b, 4, 99, "rademacher")
    assert abs(v @ w) < 5 / math.sqrt(d_b)  # independent draws


def test_gaussian_vectors_unit_norm_and_moments():
    d_b = 1 << 14
    v = rng.bath_vector(d_b, 0, 7, "gauss")
    assert abs(v @ v - 1.0) < 1e-14
    g = v * math.sqrt(d_b)
    assert abs(np.mean(g)) < 0.05 and abs(np.mean(g ** 4) - 3.0) < 0.2


def test_starting_block_layout():
    v = np.arange(1.0, 5.0)
    blk = rng.starting_block(2, v)
    assert blk.shape == (8, 2)
    np.testing.assert_array_equal(blk[:4, 0], v)
    np.testing.assert_array_equal(blk[4:, 1], v)
    assert not blk[4:, 0].any() and not blk[:4, 1].any()


# ---------------------------------------------------------------- Algorithm 1

def test_qr_drop_full_rank_matches_householder():
    z = np.random.default_rng(1).normal(size=(50, 4))
    q, r = lanczos.qr_drop(z, 1e-12, 1e-7)
    qh, rh = np.linalg.qr(z)
    s = np.sign(np.diag(rh))
    np.testing.assert_allclose(q, qh * s, atol=1e-13)
    np.testing.assert_allclose(r, rh * s[:, None], atol=1e-13)


def test_qr_drop_dependent_column():
    z = np.random.default_rng(2).normal(size=(40, 3))
    z[:, 1] = 2.0 * z[:, 0]
    q, r = lanczos.qr_drop(z, 1e-12, 1e-7)
    assert not q[:, 1].any() and r[1, 1] == 0.0 and not r[1, 2:].any()
    np.testing.assert_allclose(q @ r, z, atol=1e-12)
    np.testing.assert_allclose(q[:, [0, 2]].T @ q[:, [0, 2]], np.eye(2), atol=1e-14)


def _small_case(n=7, n_sys=1, seed=21):
    spec = W.random_model(n, n_sys, seed)
    h = spin_ops.dense_hamiltonian(spec)
    est = lanczos.Estimator(spec)
    v = est.starting_block(0, 5, "rademacher")
    return spec, h, est, v


def test_block_lanczos_invariants():
    spec, h, est, v = _small_case()
    k = 8
    qs, a_l, b_l = [], [], []
    for j, q, a, b in lanczos.block_lanczos(lambda x: h @ x, v, k, est.hnorm):
        qs.append(q)
        a_l.append(a)
        b_l.append(b)
    qn = lanczos.qr_drop(h @ qs[-1] - qs[-2] @ b_l[-2].T - qs[-1] @ a_l[-1], 0, 0)[0]
    qk = np.hstack(qs)
    t = lanczos.assemble_t(a_l, b_l)
    p = spec.d_s
    np.testing.assert_allclose(qk.T @ qk, np.eye(k * p), atol=1e-10)
    ek = np.zeros((k * p, p))
    ek[-p:, :] = np.eye(p)
    resid = h @ qk - qk @ t - qn @ b_l[-1] @ ek.T
    assert np.abs(resid).max() < 1e-11 * est.hnorm
    # A_j symmetric, B_j upper triangular with non-negative diagonal.
    for a, b in zip(a_l, b_l):
        np.testing.assert_allclose(a, a.T, atol=0)
        assert np.all(np.tril(b, -1) == 0) and np.all(np.diag(b) >= 0)


@pytest.mark.parametrize("k", [3, 5])
def test_quadrature_exact_for_polynomials_up_to_2k_minus_1(k):
    # Sec. 4.2: V^T p(H) V = E1^T p(T) E1 for deg p <= 2k-1 (block Gauss quadrature).
    spec, h, est, v = _small_case(seed=22)
    a_l, b_l = lanczos.lanczos_coefficients(lambda x: h @ x, v, k, est.hnorm)
    t = lanczos.assemble_t(a_l, b_l)
    p = spec.d_s
    hs = h / est.hnorm
    ts = t / est.hnorm
    for m in range(0, 2 * k):
        lhs = v.T @ np.linalg.matrix_power(hs, m) @ v
        rhs = np.linalg.matrix_power(ts, m)[:p, :p]
        np.testing.assert_allclose(rhs, lhs, atol=1e-12)
    m = 2 * k + 2
    lhs = v.T @ np.linalg.matrix_power(hs, m) @ v
    rhs = np.linalg.matrix_power(ts, m)[:p, :p]
    assert np.abs(rhs - lhs).max() > 1e-8  # and not beyond


@pytest.mark.parametrize("k", [4, 6])
def test_gram_form_exact_for_polynomials_up_to_k_minus_1(k):
    # Q p(T) E1 = p(H) V for deg p <= k-1 (Sec. 4.2 remark on single-vector exactness).
    spec, h, est, v = _small_case(seed=23)
    a_l, b_l = lanczos.lanczos_coefficients(lambda x: h @ x, v, k, est.hnorm)
    t = lanczos.assemble_t(a_l, b_l) / est.hnorm
    hs = h / est.hnorm
    p = spec.d_s
    for m in range(0, k):
        c = np.linalg.matrix_power(t, m)[:, :p]
        psi = lanczos.psi_gram_form(lambda x: h @ x, v, k, est.hnorm, [c])[0]
        np.testing.assert_allclose(psi, np.linalg.matrix_power(hs, m) @ v, atol=1e-11)


@pytest.mark.parametrize("n,n_sys", [(6, 1), (7, 2)])
def test_basis_estimator_equals_exact(n, n_sys):
    # Sec. 2.1: with v_l = e_l over all l the average is the partial trace itself.
    spec = W.random_model(n, n_sys, 30 + n)
    betas = [0.3, 1.0, 4.0]
    out = lanczos.Estimator(spec).run(betas, spec.d_b, k=(1 << n) // spec.d_s + 2, seed=0, dist="basis")
    rho, lnz = exact.exact_rho(spec, betas)
    np.testing.assert_allclose(out["rho"], rho, atol=1e-10)
    np.testing.assert_allclose(out["rho_quad"], rho, atol=1e-10)
    np.testing.assert_allclose(out["lnZ"], lnz, atol=1e-10)


def test_same_seed_lanczos_matches_exact_function_estimator():
    # O3 (Krylov) vs O2 (exact exp): the difference is the Krylov error only.
    spec = W.random_model(8, 1, 40)
    h = spin_ops.dense_hamiltonian(spec)
    betas = [0.5, 2.0]
    out = lanczos.Estimator(spec).run(betas, 6, k=40, seed=3, dist="gauss")
    rho2, lnz2 = lanczos.exact_function_estimator(spec, h, betas, 6, 3, "gauss")
    np.testing.assert_allclose(out["rho"], rho2, atol=1e-10)
    np.testing.assert_allclose(out["lnZ"], lnz2, atol=1e-9)


def test_e0_shift_cancels():
    spec = W.random_model(6, 1, 41)
    est = lanczos.Estimator(spec)
    a = est.run([1.0, 3.0], 4, 12, seed=1, dist="rademacher")
    b = est.run([1.0, 3.0], 4, 12, seed=1, dist="rademacher", e0=a["e0"] - 2.5)
    np.testing.assert_allclose(a["rho"], b["rho"], atol=1e-13)
    np.testing.assert_allclose(a["lnZ"], b["lnZ"], atol=1e-12)


def test_uncoupled_estimator_is_exact_for_any_vectors():
    # lambda = 0: exp(-beta H) = exp(-beta H_s) (x) exp(-beta H_b), so every
    # (I (x) v)^T ... (I (x) v) is proportional to exp(-beta H_s) (eq. HMF).
    spec = W.random_model(7, 2, 42, lam=0.0)
    out = lanczos.Estimator(spec).run([0.7, 2.0], 3, k=40, seed=9, dist="rademacher")
    for i, beta in enumerate([0.7, 2.0]):
        np.testing.assert_allclose(out["rho"][i], exact.bare_system_gibbs(spec, beta), atol=1e-10)


def test_estimator_is_unbiased_statistically():
    # Sec. 2.1 / eq. trace_est: E[(I x v)^T A (I x v)] = tr_b(A)/d_b.
    spec = W.random_model(6, 1, 43)
    beta = 0.8
    solver = exact.ExactSolver(spec)
    half = solver.exp_shifted(beta, 0.5)
    target = exact.partial_trace_bath(solver.exp_shifted(beta), spec.d_s, spec.d_b) / spec.d_b
    samples = []
    for l in range(600):
        v = rng.starting_block(spec.d_s, rng.bath_vector(spec.d_b, l, 77, "rademacher"))
        psi = half @ v
        samples.append(psi.T @ psi)
    samples = np.array(samples)
    mean = samples.mean(axis=0)
    sem = samples.std(axis=0) / math.sqrt(len(samples)) + 1e-15
    assert np.all(np.abs(mean - target) < 5 * sem)


# ---------------------------------------------------------------- post-processing

def test_entropy_special_cases():
    assert abs(post.entropy(np.eye(4) / 4) - math.log(4)) < 1e-14
    v = np.array([0.6, 0.8])
    assert abs(post.entropy(np.outer(v, v))) < 1e-14
    assert abs(post.entropy(np.diag([0.25, 0.75])) - (-(0.25 * math.log(0.25) + 0.75 * math.log(0.75)))) < 1e-15


def test_mean_force_of_gibbs_state_is_hamiltonian_plus_constant():
    spec = W.random_model(5, 2, 44, lam=0.0)
    hs = spin_ops.subsystem_hamiltonian(spec, "sys")
    beta = 1.7
    hstar = post.mean_force(exact.bare_system_gibbs(spec, beta), beta)
    diff = hstar - hs
    np.testing.assert_allclose(diff, np.trace(diff) / 4 * np.eye(4), atol=1e-12)


def test_absolute_mean_force_matches_app_c():
    n, beta = 8, 1.1
    spec = W.xy_open_chain(n, 2, 1.0, 0.3)
    rho, _ = exact.exact_rho(spec, [beta])
    hstar = post.mean_force(rho[0], beta, closed_form.log_z_star(n, beta, 1.0, 0.3))
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(hstar)),
                               np.sort(closed_form.mean_force_eigenvalues(n, beta, 1.0, 0.3)), atol=1e-12)


def test_mean_force_rejects_singular():
    with pytest.raises(ValueError):
        post.mean_force(np.diag([1.0, 0.0]), 1.0)


# ---------------------------------------------------------------- bath partition, H* constant, energy deviation

def test_mean_energy_chain_is_minus_dlnz_dbeta_and_matches_ed():
    n, beta, j, h = 6, 0.9, 1.0, 0.3
    eps = 1e-5
    num = -(closed_form.log_partition_chain(n, beta + eps, j, h)
            - closed_form.log_partition_chain(n, beta - eps, j, h)) / (2 * eps)
    assert abs(closed_form.mean_energy_chain(n, beta, j, h) - num) < 1e-8
    hm = spin_ops.dense_hamiltonian(W.xy_open_chain(n, 1, j, h))
    w = np.linalg.eigvalsh(hm)
    f = np.exp(-beta * (w - w[0]))
    assert abs(closed_form.mean_energy_chain(n, beta, j, h) - float(np.sum(w * f) / f.sum())) < 1e-12


def test_bath_spec_is_the_bare_bath():
    spec = W.random_model(7, 2, 81)
    b = W.bath_spec(spec)
    assert b.n_sites == 5 and b.n_sys == 0
    w = np.linalg.eigvalsh(spin_ops.dense_hamiltonian(b))
    for beta in (0.3, 2.0):
        ln_zb = float(np.log(np.sum(np.exp(-beta * (w - w[0])))) - beta * w[0])
        assert abs(exact.bath_log_partition(spec, beta) - ln_zb) < 1e-12


def test_energy_deviation_app_c_closed_form():
    """App. C chain, N_s = 2: tr(H* rho*) = (S(rho*) - ln Z*)/beta from the closed-form
    p_j and Z*, and tr(H_s rho_s) is the mean energy of the 2-site chain."""
    n, beta, j, h = 8, 1.3, 1.0, 0.3
    spec = W.xy_open_chain(n, 2, j, h)
    rho, _ = exact.exact_rho(spec, [beta])
    hstar = post.mean_force(rho[0], beta, closed_form.log_z_star(n, beta, j, h))
    hs = np.real(spin_ops.subsystem_hamiltonian(spec, "sys"))
    got = post.energy_deviation(rho[0], hstar, hs, beta)
    p = closed_form.rho_eigenvalues(n, beta, j, h)
    s = float(-np.sum(p * np.log(p)))
    want = (s - closed_form.log_z_star(n, beta, j, h)) / beta - closed_form.mean_energy_chain(2, beta, j, h)
    assert abs(got - want) < 1e-12


def test_energy_deviation_vanishes_without_coupling():
    """lambda = 0: H_t = H_s + H_b, so Z_t = Z_s Z_b, H* = H_s and the deviation is 0."""
    spec = W.random_model(7, 1, 82, lam=0.0)
    beta = 0.8
    rho, lnz = exact.exact_rho(spec, [beta])
    ln_zb = exact.bath_log_partition(spec, beta)
    hs = np.real(spin_ops.subsystem_hamiltonian(spec, "sys"))
    ws = np.linalg.eigvalsh(hs)
    ln_zs = float(np.log(np.sum(np.exp(-beta * (ws - ws[0])))) - beta * ws[0])
    assert abs(lnz[0] - (ln_zs + ln_zb)) < 1e-11
    hstar = post.mean_force(rho[0], beta, lnz[0] - ln_zb)
    np.testing.assert_allclose(hstar, hs, atol=1e-11)
    assert abs(post.energy_deviation(rho[0], hstar, hs, beta)) < 1e-11


# ---------------------------------------------------------------- per-vector (block size 1) Lanczos

def test_single_vector_lanczos_converges_to_exact_function_estimator():
    """Sec. 4.2: regular Lanczos on each column e_i (x) v_l, Gram form with the cross
    terms psi_i^T psi_j; at large k it equals eq. rho_est with the exact exp(-beta H/2)."""
    spec = W.random_model(8, 2, 5)
    betas = [0.5, 2.0]
    s = lanczos.Estimator(spec).run(betas, 6, 30, 3, "gauss", block=False)
    h = spin_ops.dense_hamiltonian(spec)
    rho2, lnz2 = lanczos.exact_function_estimator(spec, h, betas, 6, 3, "gauss")
    np.testing.assert_allclose(s["rho"], rho2, atol=1e-9)
    np.testing.assert_allclose(s["lnZ"], lnz2, atol=1e-9)
    # the cross terms carry information: zeroing them changes rho
    assert np.abs(rho2[0] - np.diag(np.diag(rho2[0]))).max() > 1e-3


def test_single_vector_equals_block_for_one_system_state():
    spec = W.random_model(7, 0, 6)
    b = lanczos.Estimator(spec).run([1.0], 5, 12, 4, "rademacher")
    s = lanczos.Estimator(spec).run([1.0], 5, 12, 4, "rademacher", block=False)
    np.testing.assert_allclose(s["gram_l"], b["gram_l"], rtol=1e-13, atol=0)
    np.testing.assert_allclose(s["lnZ"], b["lnZ"], rtol=1e-13, atol=0)


def test_single_vector_exhaustive_is_exact():
    spec = W.random_model(6, 1, 7)
    betas = [0.4, 3.0]
    s = lanczos.Estimator(spec).run(betas, spec.d_b, spec.dim + 2, 0, "basis", block=False)
    rho, lnz = exact.exact_rho(spec, betas)
    np.testing.assert_allclose(s["rho"], rho, atol=1e-10)
    np.testing.assert_allclose(s["lnZ"], lnz, atol=1e-9)


def test_block_lanczos_more_accurate_than_single_at_equal_k():
    """The paper's remark (Sec. 4.2): at equal k block Lanczos is exact to a higher
    polynomial degree; on this model its error is smaller at every k tried."""
    spec = W.random_model(8, 2, 5)
    h = spin_ops.dense_hamiltonian(spec)
    rho2, _ = lanczos.exact_function_estimator(spec, h, [2.0], 6, 3, "gauss")
    for k in (4, 6, 8):
        b = lanczos.Estimator(spec).run([2.0], 6, k, 3, "gauss")
        s = lanczos.Estimator(spec).run([2.0], 6, k, 3, "gauss", block=False)
        assert np.abs(b["rho"] - rho2).max() < np.abs(s["rho"] - rho2).max()


@pytest.mark.parametrize("maker", [lambda: W.random_model(7, 2, 5), lambda: W.long_range_xxz(8, 1, 1.0, 0.5, 0.3),
                                   lambda: W.long_range_tfim(7, 2, 1.5, 0.9, lam=0.4), lambda: W.xxz_chain(8, 1)])
def test_hamiltonian_row_is_the_kronecker_row(maker):
    """Every row of the single-row construction (Pauli action on one basis vector) equals
    the row of the Kronecker-built sparse H, with no extra entries: random anisotropic
    couplings with fields and lambda, long-range XXZ, long-range TFIM, the NN chain."""
    spec = maker()
    h = spin_ops.sparse_hamiltonian(spec).tocsr()
    for s in range(1 << spec.n_sites):
        row = spin_ops.hamiltonian_row(spec, s)
        dense = h.getrow(s).toarray().ravel()
        got = np.zeros_like(dense)
        for col, v in row.items():
            got[col] += v
        np.testing.assert_allclose(got, dense, atol=1e-13, rtol=0)
