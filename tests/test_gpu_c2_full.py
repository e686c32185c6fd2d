"""Full-length oracle parity of the benchmark configuration.

Long-range transverse-field Ising model, N = 22 (D = 2^22), N_s = 2, n_v = 32 normalised
Gaussian bath vectors (seed 20220418), k = 60, beta = 1 -- the launch configuration the
benchmark times (all 32 vectors in one 128-column block). The oracle (Algorithm 1 in
float64 NumPy, eqs. trB_est and rho_est) cannot run all 32 vectors in a test's time,
but the estimator is a sum over bath vectors, so the per-vector results of sampled
vectors l are checked element by element against the oracle run on those vectors
alone, with the GPU's shift E0:

  * the Gram form G_l = psi_l^T psi_l and the quadrature form E1^T exp(-beta (T_l - E0)) E1
    after all 60 steps: max |G^gpu - G^oracle| <= tol * tr G^oracle, tol = 1e-10 (float64
    path) and 1e-4 (float32 path), the precision contract of rho*;
  * the coefficients A_j, B_j while the basis is still orthogonal: max deviation
    <= 1e-9 ||H||_bound (float64) and 1e-4 ||H||_bound (float32). Once a Ritz value
    has converged, finite-precision Lanczos loses orthogonality (Sec. 4.3) and the
    later coefficients depend on the rounding of each implementation -- two correct
    runs differ there while f(T) still agrees, which is what the first check pins.
    The loss of orthogonality grows in proportion to the unit roundoff u of the
    arithmetic, so the oracle's float64 basis (loss ||Q_1^T Q_j||) marks the horizon
    of both runs: float64 steps with loss <= 1e-8, float32 steps with loss <= 100 u_64
    (where a float32 basis has lost at most about 100 u_32 = 6e-6).

The oracle runs in worker processes started with `spawn` (one per sampled vector).
"""
import json
import multiprocessing as mp
import os

import numpy as np
import pytest

import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

SAMPLED = (0, 31)
TOL_FORM = {"fp64": 1e-10, "fp32": 1e-4}
TOL_T = {"fp64": 1e-9, "fp32": 1e-4}
ORTHO = {"fp64": 1e-8, "fp32": 100 * 2.0 ** -53}


def _oracle_vector(args):
    """Oracle run of bath vector l of the c2 workload (g index 0) with shift e0: the
    coefficients of Algorithm 1 with ||Q_1^T Q_j|| per step, then both forms."""
    l, e0 = args
    from oracle import lanczos, spin_ops
    c = W.config_c2(0)
    ham = spin_ops.TensorHamiltonian(c["spec"])
    est = lanczos.Estimator(c["spec"], apply_h=ham, hnorm=ham.norm_bound())
    v = est.starting_block(l, c["seed"], c["dist"])
    a_l, b_l, ortho = [], [], []
    for _, q, a, b in lanczos.block_lanczos(est.apply_h, v, c["k"], est.hnorm):
        a_l.append(a)
        b_l.append(b)
        ortho.append(float(np.linalg.norm(v.T @ q, 2)) if ortho else 0.0)
    t = lanczos.assemble_t(a_l, b_l)
    p = v.shape[1]
    beta = float(c["betas"][0])
    cf = lanczos.function_of_t_first_block(t, p, lambda x: np.exp(-beta * (x - e0) / 2.0))
    psi = lanczos.psi_gram_form(est.apply_h, v, c["k"], est.hnorm, [cf])[0]
    return dict(gram=psi.T @ psi, quad=cf.T @ cf, t_a=np.array(a_l), t_b=np.array(b_l),
                ortho=np.array(ortho), hnorm=est.hnorm)


@pytest.fixture(scope="module")
def gpu_runs(lib):
    c = W.config_c2(0)
    ctx = lib.Context(0)
    ham = lib.Hamiltonian(ctx, c["spec"])
    out = {}
    for prec in ("fp32", "fp64"):
        out[prec] = ham.estimate(c["betas"], c["n_v"], c["k"], c["seed"], precision=prec, dist=c["dist"],
                                 full=True)
    ham.close()
    ctx.close()
    return out


@pytest.fixture(scope="module")
def oracle_runs(gpu_runs):
    e0 = gpu_runs["fp64"]["e0"]
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS"):
        os.environ.setdefault(var, "4")
    with mp.get_context("spawn").Pool(len(SAMPLED)) as pool:
        res = pool.map(_oracle_vector, [(l, e0) for l in SAMPLED], chunksize=1)
    return e0, dict(zip(SAMPLED, res))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_c2_full_length_per_vector_gram_and_coefficients(gpu_runs, oracle_runs, prec):
    e0_ref, ref = oracle_runs
    out = gpu_runs[prec]
    c = W.config_c2(0)
    beta = float(c["betas"][0])
    report = {"prec": prec, "e0_gpu": out["e0"], "e0_fp64": e0_ref}
    ok = True
    for l in SAMPLED:
        r = ref[l]
        # The oracle ran with the float64 path's E0; both forms scale as exp(beta E0).
        scale = np.exp(beta * (out["e0"] - e0_ref))
        dev = {}
        for name, got, want in (("gram", out["gram_l"][0, l], r["gram"] * scale),
                                ("quad", out["quad_l"][0, l], r["quad"] * scale)):
            dev[name] = float(np.abs(got - want).max() / np.trace(want))
            ok &= dev[name] <= TOL_FORM[prec]
        steps = int(np.sum(np.cumprod(r["ortho"] <= ORTHO[prec])))  # leading steps still orthogonal
        da = np.abs(out["t_a"][l] - r["t_a"]).max(axis=(1, 2)) / r["hnorm"]
        db = np.abs(out["t_b"][l] - r["t_b"]).max(axis=(1, 2)) / r["hnorm"]
        dev.update(orthogonal_steps=steps, t_a_rel_hnorm=float(da[:steps].max()),
                   t_b_rel_hnorm=float(db[:steps].max()),
                   ortho_loss=[float(x) for x in r["ortho"][::6]],
                   t_dev_every_6th_step=[float(max(x, y)) for x, y in zip(da[::6], db[::6])])
        ok &= steps >= 10 and dev["t_a_rel_hnorm"] <= TOL_T[prec] and dev["t_b_rel_hnorm"] <= TOL_T[prec]
        report[f"l{l}"] = dev
    print("c2 full-length parity:", json.dumps(report))
    assert ok, report
