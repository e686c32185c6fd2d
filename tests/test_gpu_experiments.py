"""The solvable-chain experiment of Sec. 5.1 (Fig. 1) against the closed form of App. C.

Open isotropic XY chain of N = 18 spins (coefficient J/2 on XX + YY, (h/2) Z with
h = 0.3 J; the convention under which App. C holds), system = the first two spins,
k = 30 block-Lanczos steps, n_v = 100 bath vectors drawn uniformly from the unit sphere
(normalised Gaussian), 100 independent runs (seeds). Sec. 5.1 reports the median and
the 10%/90% quantiles of the eigenvalues of rho*(beta) and of H*(beta) (with its
constant, eq. H_est: ln Z_b from the bare bath with the same vectors) over the runs.
The chain is far beyond exact diagonalisation (D = 2^18), so the reference is the
closed form alone. Checks, per beta and eigenvalue:

  * the median of the runs is within a quarter of the 10-90% spread (about 2.5
    standard errors of a median of 100 runs) plus 2e-3 of the exact value: the
    estimator is unbiased up to the Krylov error, which is small at k = 30;
  * the exact value lies inside the 10-90% band widened by that same margin.

The float32 path (the production precision) is used; the table is printed as JSON.
"""
import json

import numpy as np
import pytest

import workloads as W
from oracle import closed_form

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N, N_S, H_FIELD, K, N_V, RUNS = 18, 2, 0.3, 30, 100, 100
BETAS = W.beta_grid(12, 0.1, 10.0)


def test_e1_solvable_chain_matches_app_c(lib):
    spec = W.xy_open_chain(N, N_S, 1.0, H_FIELD)
    ctx = lib.Context(0)
    try:
        tot = lib.Hamiltonian(ctx, spec)
        bath = lib.Hamiltonian(ctx, spec, part="bath")
        p_runs = np.zeros((RUNS, len(BETAS), 4))
        h_runs = np.zeros((RUNS, len(BETAS), 4))
        for r in range(RUNS):
            seed = 20220500 + r
            rt = tot.estimate(BETAS, N_V, K, seed, precision="fp32", dist="gauss")
            rb = bath.estimate(BETAS, N_V, K, seed, precision="fp32", dist="gauss")
            for i, beta in enumerate(BETAS):
                p_runs[r, i] = np.sort(np.linalg.eigvalsh(rt["rho"][i]))
                hs = lib.mean_force_abs(rt["rho"][i], beta, rt["lnZ"][i], rb["lnZ"][i])
                h_runs[r, i] = np.sort(np.linalg.eigvalsh(hs))[::-1]  # matches ascending p
        tot.close()
        bath.close()
    finally:
        ctx.close()
    table, bad = [], []
    for name, runs, exact_of in (("rho", p_runs, closed_form.rho_eigenvalues),
                                 ("hstar", h_runs, closed_form.mean_force_eigenvalues)):
        q10, med, q90 = np.percentile(runs, [10, 50, 90], axis=0)
        for i, beta in enumerate(BETAS):
            exact = exact_of(N, float(beta), 1.0, H_FIELD)
            margin = 0.25 * (q90[i] - q10[i]) + 2e-3 * np.maximum(1.0, np.abs(exact))
            table.append({"quantity": name, "beta": float(beta), "exact": exact.tolist(),
                          "median": med[i].tolist(), "q10": q10[i].tolist(), "q90": q90[i].tolist()})
            if np.any(np.abs(med[i] - exact) > margin):
                bad.append((name, float(beta), "median", (med[i] - exact).tolist(), margin.tolist()))
            if np.any(exact < q10[i] - margin) or np.any(exact > q90[i] + margin):
                bad.append((name, float(beta), "band", exact.tolist(), q10[i].tolist(), q90[i].tolist()))
    print("E1 table:", json.dumps(table))
    assert not bad, bad
