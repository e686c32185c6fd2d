// Host float64 dense symmetric eigensolver and the post-processing of rho*.
//
// The small dense step of the estimator (eq. fT: f(T_l) from the eigen-
// decomposition of the block tridiagonal T_l, Sec. 3.1 "T_l can be diagonalized
// exactly") and H* through the eigenvalues of rho* (end of Sec. 3.2) both need
// eigenpairs of small symmetric matrices. Method (textbook, Golub & Van Loan,
// "Matrix Computations", Sec. 8.3): Householder reduction to tridiagonal form with
// the orthogonal factor accumulated, then implicit symmetric QR steps with the
// Wilkinson shift, rotations accumulated into the eigenvector matrix.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <numeric>
#include <vector>

#include "rdm_internal.h"

namespace rdm {
void set_error(const char* fmt, ...);

// Eigen-decomposition of the symmetric n x n row-major matrix `a`.
// w: ascending eigenvalues; vt (optional): n*n with ROW j = eigenvector j.
// Returns false if the QR iteration did not converge.
bool sym_eig(int n, const double* a_in, double* w, double* vt) {
  if (n <= 0) return true;
  if (n == 1) {
    w[0] = a_in[0];
    if (vt) vt[0] = 1.0;
    return true;
  }
  std::vector<double> a(a_in, a_in + (size_t)n * n);
  const bool want = vt != nullptr;
  // qt[j*n + r] = Q[r][j]: column j of Q stored contiguously.
  std::vector<double> qt;
  if (want) {
    qt.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) qt[(size_t)i * n + i] = 1.0;
  }
  std::vector<double> v(n), p(n), wv(n), t(n);
  auto A = [&](int i, int j) -> double& { return a[(size_t)i * n + j]; };

  // ---- Householder tridiagonalisation: Q^T A Q = tridiag.
  for (int k = 0; k + 2 < n; ++k) {
    double tail = 0.0;
    for (int i = k + 2; i < n; ++i) tail += A(i, k) * A(i, k);
    if (tail == 0.0) continue;
    const double x0 = A(k + 1, k);
    const double nrm = std::sqrt(tail + x0 * x0);
    const double alpha = x0 > 0 ? -nrm : nrm;
    v[k + 1] = x0 - alpha;
    double vv = v[k + 1] * v[k + 1];
    for (int i = k + 2; i < n; ++i) {
      v[i] = A(i, k);
      vv += v[i] * v[i];
    }
    const double beta = 2.0 / vv;
    double vp = 0.0;
    for (int i = k + 1; i < n; ++i) {
      double s = 0.0;
      for (int j = k + 1; j < n; ++j) s += A(i, j) * v[j];
      p[i] = beta * s;
      vp += v[i] * p[i];
    }
    const double kk = 0.5 * beta * vp;
    for (int i = k + 1; i < n; ++i) wv[i] = p[i] - kk * v[i];
    for (int i = k + 1; i < n; ++i)
      for (int j = k + 1; j < n; ++j) A(i, j) -= v[i] * wv[j] + wv[i] * v[j];
    A(k + 1, k) = A(k, k + 1) = alpha;
    for (int i = k + 2; i < n; ++i) A(i, k) = A(k, i) = 0.0;
    if (want) {
      // Q <- Q (I - beta v v^T) on columns k+1..n-1.
      std::fill(t.begin(), t.end(), 0.0);
      for (int j = k + 1; j < n; ++j) {
        const double vj = v[j];
        const double* qj = &qt[(size_t)j * n];
        for (int r = 0; r < n; ++r) t[r] += qj[r] * vj;
      }
      for (int j = k + 1; j < n; ++j) {
        const double f = beta * v[j];
        double* qj = &qt[(size_t)j * n];
        for (int r = 0; r < n; ++r) qj[r] -= f * t[r];
      }
    }
  }
  std::vector<double> d(n), e(n, 0.0);
  for (int i = 0; i < n; ++i) d[i] = A(i, i);
  for (int i = 0; i + 1 < n; ++i) e[i] = A(i + 1, i);

  // ---- implicit symmetric QR with Wilkinson shift on (d, e).
  const double eps = DBL_EPSILON;
  int hi = n - 1;
  long iters = 0;
  const long max_iters = 60L * n;
  while (hi > 0) {
    if (std::fabs(e[hi - 1]) <= eps * (std::fabs(d[hi - 1]) + std::fabs(d[hi])) ||
        std::fabs(e[hi - 1]) < DBL_MIN) {
      e[hi - 1] = 0.0;
      --hi;
      continue;
    }
    int lo = hi - 1;
    while (lo > 0 && std::fabs(e[lo - 1]) > eps * (std::fabs(d[lo - 1]) + std::fabs(d[lo])) &&
           std::fabs(e[lo - 1]) >= DBL_MIN)
      --lo;
    if (++iters > max_iters) return false;
    const double delta = 0.5 * (d[hi - 1] - d[hi]);
    const double eh = e[hi - 1];
    const double denom = delta + (delta >= 0 ? 1.0 : -1.0) * std::hypot(delta, eh);
    const double mu = d[hi] - eh * eh / denom;
    double x = d[lo] - mu;
    double z = e[lo];
    for (int k = lo; k < hi; ++k) {
      const double r = std::hypot(x, z);
      const double c = r == 0.0 ? 1.0 : x / r;
      const double s = r == 0.0 ? 0.0 : -z / r;
      if (k > lo) e[k - 1] = r;
      const double dk = d[k], dk1 = d[k + 1], ek = e[k];
      d[k] = c * c * dk - 2.0 * c * s * ek + s * s * dk1;
      d[k + 1] = s * s * dk + 2.0 * c * s * ek + c * c * dk1;
      e[k] = c * s * (dk - dk1) + (c * c - s * s) * ek;
      if (k + 1 < hi) {
        x = e[k];
        z = -s * e[k + 1];
        e[k + 1] = c * e[k + 1];
      }
      if (want) {
        double* qa = &qt[(size_t)k * n];
        double* qb = &qt[(size_t)(k + 1) * n];
        for (int rr = 0; rr < n; ++rr) {
          const double ya = qa[rr], yb = qb[rr];
          qa[rr] = c * ya - s * yb;
          qb[rr] = s * ya + c * yb;
        }
      }
    }
  }
  // ---- sort ascending.
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int x1, int x2) { return d[x1] < d[x2]; });
  for (int j = 0; j < n; ++j) w[j] = d[idx[j]];
  if (want)
    for (int j = 0; j < n; ++j)
      std::copy(&qt[(size_t)idx[j] * n], &qt[(size_t)idx[j] * n] + n, &vt[(size_t)j * n]);
  return true;
}


// sqrt(x^2 + z^2): the plain formula where the squares can neither overflow nor
// underflow, std::hypot (slower, scaled) elsewhere.
static inline double rot_norm(double x, double z) {
  const double m = std::max(std::fabs(x), std::fabs(z));
  if (m > 1e-150 && m < 1e150) return std::sqrt(x * x + z * z);
  return std::hypot(x, z);
}

// f(T) E1 for every beta of a grid without forming eigenvectors.
//
// T = Q S Q^T with S tridiagonal, S = U Theta U^T (implicit QR, U = G_1 G_2 ... kept
// as rotations). Then
//   c_beta = Q U exp(-beta (Theta - t_min)/2) U^T Q^T E1,
// applied to the p columns of E1 only instead of accumulating full eigenvectors.
// Q comes from one of two reductions to tridiagonal form:
//  * T banded with semi-bandwidth b < n - 2 (the block tridiagonal T_l of Algorithm 1
//    has b = d_s): Givens rotations that zero the band column by column and chase
//    each bulge they create down the band (Schwarz's band reduction, Golub & Van Loan
//    Sec. 8.3 notes), O(n^2 b) work; Q = R_1^T R_2^T ... kept as rotations.
//  * otherwise Householder reflectors, O(n^3); Q = H_0 H_1 ... kept as reflectors.
// The shift is this matrix's own smallest eigenvalue t_min (no overflow); the caller
// rescales by exp(-beta (t_min - E0)/2) once the common E0 is known.
bool tdense_fT(int n, int p, const double* t_in, int n_beta, const double* betas, double* t_min,
               double* c_out) {
  std::vector<double> a(t_in, t_in + (size_t)n * n);
  auto A = [&](int i, int j) -> double& { return a[(size_t)i * n + j]; };
  std::vector<double> hv, hb;  // Householder reflector k: v in row k, beta
  std::vector<double> p_(n), wv(n);
  int band = 0;  // semi-bandwidth of T
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j)
      if (A(i, j) != 0.0 || A(j, i) != 0.0) band = std::max(band, i - j);
  const bool banded = band >= 2 && band < n - 2;
  // y = Q^T E1 (n x p, row-major), built alongside the reduction.
  std::vector<double> y((size_t)n * p, 0.0);
  for (int i = 0; i < p && i < n; ++i) y[(size_t)i * p + i] = 1.0;
  struct BandRot {
    int q;  // plane (q - 1, q)
    double c, s;
  };
  std::vector<BandRot> brots;
  if (banded) {
    // Rotation R in plane (q-1, q) with rows (c s; -s c): A <- R A R^T, y <- R y. Rows
    // and columns q-1, q are nonzero only within band + 1 of the diagonal (the bulge),
    // so only that window is touched.
    auto rotate = [&](int q, double c, double s) {
      const int pr = q - 1;
      const int lo = std::max(0, pr - band - 2), hi = std::min(n, q + band + 3);
      double* rp = &a[(size_t)pr * n];
      double* rq = &a[(size_t)q * n];
      for (int j = lo; j < hi; ++j) {
        const double u = rp[j], w = rq[j];
        rp[j] = c * u + s * w;
        rq[j] = -s * u + c * w;
      }
      for (int i = lo; i < hi; ++i) {
        double* ri = &a[(size_t)i * n];
        const double u = ri[pr], w = ri[q];
        ri[pr] = c * u + s * w;
        ri[q] = -s * u + c * w;
      }
      double* yp = &y[(size_t)pr * p];
      double* yq = &y[(size_t)q * p];
      for (int t = 0; t < p; ++t) {
        const double u = yp[t], w = yq[t];
        yp[t] = c * u + s * w;
        yq[t] = -s * u + c * w;
      }
      brots.push_back(BandRot{q, c, s});
    };
    for (int k = 0; k + 2 < n; ++k) {
      for (int l = std::min(band, n - 1 - k); l >= 2; --l) {
        // zero A(k + l, k) from row k + l - 1, then chase the bulge it leaves at
        // (i + band, i - 1) down the band until it leaves the matrix
        int i = k + l, col = k;
        while (true) {
          const double x = A(i - 1, col), z = A(i, col);
          if (z != 0.0) {
            const double r = rot_norm(x, z);
            rotate(i, x / r, z / r);
            A(i, col) = A(col, i) = 0.0;
          }
          if (i + band >= n) break;
          col = i - 1;
          i += band;
        }
      }
    }
  } else {
    hv.assign((size_t)n * n, 0.0);
    hb.assign(n, 0.0);
  }
  for (int k = 0; !banded && k + 2 < n; ++k) {
    double tail = 0.0;
    for (int i = k + 2; i < n; ++i) tail += A(i, k) * A(i, k);
    if (tail == 0.0) continue;
    const double x0 = A(k + 1, k);
    const double nrm = std::sqrt(tail + x0 * x0);
    const double alpha = x0 > 0 ? -nrm : nrm;
    double* v = &hv[(size_t)k * n];
    v[k + 1] = x0 - alpha;
    double vv = v[k + 1] * v[k + 1];
    for (int i = k + 2; i < n; ++i) {
      v[i] = A(i, k);
      vv += v[i] * v[i];
    }
    const double beta = 2.0 / vv;
    hb[k] = beta;
    double vp = 0.0;
    for (int i = k + 1; i < n; ++i) {
      double sacc = 0.0;
      const double* ai = &a[(size_t)i * n];
      for (int j = k + 1; j < n; ++j) sacc += ai[j] * v[j];
      p_[i] = beta * sacc;
      vp += v[i] * p_[i];
    }
    const double kk = 0.5 * beta * vp;
    for (int i = k + 1; i < n; ++i) wv[i] = p_[i] - kk * v[i];
    for (int i = k + 1; i < n; ++i) {
      double* ai = &a[(size_t)i * n];
      for (int j = k + 1; j < n; ++j) ai[j] -= v[i] * wv[j] + wv[i] * v[j];
    }
    A(k + 1, k) = A(k, k + 1) = alpha;
    for (int i = k + 2; i < n; ++i) A(i, k) = A(k, i) = 0.0;
  }
  std::vector<double> d(n), e(n, 0.0);
  for (int i = 0; i < n; ++i) d[i] = A(i, i);
  for (int i = 0; i + 1 < n; ++i) e[i] = A(i + 1, i);
  // Householder case: y = Q^T E1 by applying H_0, H_1, ... in order.
  auto apply_reflector = [&](int k, std::vector<double>& z) {
    if (hb[k] == 0.0) return;
    const double* v = &hv[(size_t)k * n];
    for (int c = 0; c < p; ++c) {
      double dot = 0.0;
      for (int i = k + 1; i < n; ++i) dot += v[i] * z[(size_t)i * p + c];
      dot *= hb[k];
      for (int i = k + 1; i < n; ++i) z[(size_t)i * p + c] -= dot * v[i];
    }
  };
  if (!banded)
    for (int k = 0; k + 2 < n; ++k) apply_reflector(k, y);
  // Implicit QR with Wilkinson shift; each rotation is also applied to y (U^T y).
  struct Rot {
    int k;
    double c, s;
  };
  std::vector<Rot> rots;
  rots.reserve((size_t)4 * n * n / 2 + 16);
  auto rot_t = [&](std::vector<double>& z, int k, double c, double sn) {  // G^T z
    double* za = &z[(size_t)k * p];
    double* zb = &z[(size_t)(k + 1) * p];
    for (int q = 0; q < p; ++q) {
      const double u = za[q], w = zb[q];
      za[q] = c * u - sn * w;
      zb[q] = sn * u + c * w;
    }
  };
  const double eps = DBL_EPSILON;
  int hi = n - 1;
  long iters = 0;
  const long max_iters = 60L * n;
  while (hi > 0) {
    if (std::fabs(e[hi - 1]) <= eps * (std::fabs(d[hi - 1]) + std::fabs(d[hi])) ||
        std::fabs(e[hi - 1]) < DBL_MIN) {
      e[hi - 1] = 0.0;
      --hi;
      continue;
    }
    int lo = hi - 1;
    while (lo > 0 && std::fabs(e[lo - 1]) > eps * (std::fabs(d[lo - 1]) + std::fabs(d[lo])) &&
           std::fabs(e[lo - 1]) >= DBL_MIN)
      --lo;
    if (++iters > max_iters) return false;
    const double delta = 0.5 * (d[hi - 1] - d[hi]);
    const double eh = e[hi - 1];
    const double denom = delta + (delta >= 0 ? 1.0 : -1.0) * std::hypot(delta, eh);
    const double mu = d[hi] - eh * eh / denom;
    double x = d[lo] - mu;
    double z = e[lo];
    for (int k = lo; k < hi; ++k) {
      const double r = rot_norm(x, z);
      const double c = r == 0.0 ? 1.0 : x / r;
      const double sn = r == 0.0 ? 0.0 : -z / r;
      if (k > lo) e[k - 1] = r;
      const double dk = d[k], dk1 = d[k + 1], ek = e[k];
      d[k] = c * c * dk - 2.0 * c * sn * ek + sn * sn * dk1;
      d[k + 1] = sn * sn * dk + 2.0 * c * sn * ek + c * c * dk1;
      e[k] = c * sn * (dk - dk1) + (c * c - sn * sn) * ek;
      if (k + 1 < hi) {
        x = e[k];
        z = -sn * e[k + 1];
        e[k + 1] = c * e[k + 1];
      }
      rots.push_back(Rot{k, c, sn});
      rot_t(y, k, c, sn);
    }
  }
  double tmin = d[0];
  for (int i = 1; i < n; ++i) tmin = std::min(tmin, d[i]);
  *t_min = tmin;
  // For every beta: z_beta = exp(-beta (theta - t_min)/2) * y, then U z (rotations in
  // reverse, untransposed), then Q z. All betas go through the rotations together: row m
  // of Z holds the p columns of every beta (width p * n_beta), so each rotation is one
  // contiguous loop; every element sees the same operations as one beta alone.
  const int w = p * n_beta;
  std::vector<double> zb((size_t)n * w);
  for (int m = 0; m < n; ++m)
    for (int b = 0; b < n_beta; ++b) {
      const double f = std::exp(-0.5 * betas[b] * (d[m] - tmin));
      for (int q = 0; q < p; ++q) zb[(size_t)m * w + b * p + q] = f * y[(size_t)m * p + q];
    }
  for (size_t r = rots.size(); r-- > 0;) {
    const Rot& g = rots[r];
    double* za = &zb[(size_t)g.k * w];
    double* zc = &zb[(size_t)(g.k + 1) * w];
    for (int q = 0; q < w; ++q) {
      const double u = za[q], v = zc[q];
      za[q] = g.c * u + g.s * v;
      zc[q] = -g.s * u + g.c * v;
    }
  }
  if (banded) {  // Q z = R_1^T ... R_m^T z: transposed rotations in reverse order
    for (size_t r = brots.size(); r-- > 0;) {
      const BandRot& g = brots[r];
      double* za = &zb[(size_t)(g.q - 1) * w];
      double* zc = &zb[(size_t)g.q * w];
      for (int q = 0; q < w; ++q) {
        const double u = za[q], v = zc[q];
        za[q] = g.c * u - g.s * v;
        zc[q] = g.s * u + g.c * v;
      }
    }
  }
  if (!banded) {
    for (int k = n - 3; k >= 0; --k) {
      if (hb[k] == 0.0) continue;
      const double* v = &hv[(size_t)k * n];
      for (int c = 0; c < w; ++c) {
        double dot = 0.0;
        for (int i = k + 1; i < n; ++i) dot += v[i] * zb[(size_t)i * w + c];
        dot *= hb[k];
        for (int i = k + 1; i < n; ++i) zb[(size_t)i * w + c] -= dot * v[i];
      }
    }
  }
  for (int b = 0; b < n_beta; ++b)
    for (int m = 0; m < n; ++m)
      for (int q = 0; q < p; ++q) c_out[((size_t)b * n + m) * p + q] = zb[(size_t)m * w + b * p + q];
  return true;
}

}  // namespace rdm

using rdm::set_error;

extern "C" rdm_status rdm_function_of_t(int n, int p, const double* t, int n_beta, const double* betas,
                                        double* t_min, double* c) {
  if (n < 1 || n > 8192 || p < 1 || p > n || n_beta < 1 || !t || !betas || !t_min || !c) {
    set_error("rdm_function_of_t: need 1 <= p <= n <= 8192, n_beta >= 1 and non-NULL arrays");
    return RDM_EINVAL;
  }
  for (int b = 0; b < n_beta; ++b)
    if (!(betas[b] >= 0.0) || !std::isfinite(betas[b])) {
      set_error("rdm_function_of_t: beta[%d] must be finite and >= 0", b);
      return RDM_EINVAL;
    }
  for (size_t i = 0; i < (size_t)n * n; ++i)
    if (!std::isfinite(t[i])) {
      set_error("rdm_function_of_t: T has a non-finite entry");
      return RDM_EINVAL;
    }
  if (!rdm::tdense_fT(n, p, t, n_beta, betas, t_min, c)) {
    set_error("rdm_function_of_t: QR iteration did not converge");
    return RDM_ENUMERIC;
  }
  return RDM_OK;
}

extern "C" rdm_status rdm_symmetric_eig(int n, const double* a, double* w, double* v) {
  if (n < 1 || n > 8192 || !a || !w) {
    set_error("rdm_symmetric_eig: need 1 <= n <= 8192 and non-NULL a, w");
    return RDM_EINVAL;
  }
  std::vector<double> vt;
  if (v) vt.resize((size_t)n * n);
  if (!rdm::sym_eig(n, a, w, v ? vt.data() : nullptr)) {
    set_error("rdm_symmetric_eig: QR iteration did not converge");
    return RDM_ENUMERIC;
  }
  if (v)
    for (int r = 0; r < n; ++r)
      for (int j = 0; j < n; ++j) v[(size_t)r * n + j] = vt[(size_t)j * n + r];
  return RDM_OK;
}

static bool symmetrised(const double* rho, int d, std::vector<double>& out) {
  out.resize((size_t)d * d);
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      const double x = 0.5 * (rho[i * d + j] + rho[j * d + i]);
      if (!std::isfinite(x)) return false;
      out[i * d + j] = x;
    }
  return true;
}

extern "C" rdm_status rdm_mean_force(const double* rho, int d_s, double beta, double* h_out) {
  if (!rho || !h_out || d_s < 1 || d_s > 64 || !(beta > 0) || !std::isfinite(beta)) {
    set_error("rdm_mean_force: need rho, h_out, 1 <= d_s <= 64 and finite beta > 0");
    return RDM_EINVAL;
  }
  std::vector<double> a, w(d_s), vt((size_t)d_s * d_s);
  if (!symmetrised(rho, d_s, a)) {
    set_error("rdm_mean_force: rho has non-finite entries");
    return RDM_ENUMERIC;
  }
  if (!rdm::sym_eig(d_s, a.data(), w.data(), vt.data())) {
    set_error("rdm_mean_force: eigensolver did not converge");
    return RDM_ENUMERIC;
  }
  for (int j = 0; j < d_s; ++j)
    if (!(w[j] > 0)) {
      set_error("rdm_mean_force: rho has eigenvalue %.3e <= 0, ln(rho) undefined", w[j]);
      return RDM_ENOTPD;
    }
  // H = -(1/beta) U diag(ln p) U^T
  for (int r = 0; r < d_s; ++r)
    for (int c = 0; c < d_s; ++c) {
      double s = 0.0;
      for (int j = 0; j < d_s; ++j) s += vt[j * d_s + r] * std::log(w[j]) * vt[j * d_s + c];
      h_out[r * d_s + c] = -s / beta;
    }
  return RDM_OK;
}

extern "C" rdm_status rdm_mean_force_abs(const double* rho, int d_s, double beta, double ln_z_t,
                                         double ln_z_b, double* h_out) {
  if (!std::isfinite(ln_z_t) || !std::isfinite(ln_z_b)) {
    set_error("rdm_mean_force_abs: ln_z_t and ln_z_b must be finite");
    return RDM_EINVAL;
  }
  const rdm_status st = rdm_mean_force(rho, d_s, beta, h_out);
  if (st != RDM_OK) return st;
  // -(1/beta) ln(Z_t rho / Z_b) = -(1/beta) ln rho - (1/beta)(ln Z_t - ln Z_b) I
  const double shift = (ln_z_t - ln_z_b) / beta;
  for (int r = 0; r < d_s; ++r) h_out[r * d_s + r] -= shift;
  return RDM_OK;
}

extern "C" rdm_status rdm_energy_deviation(const double* rho, const double* h_star, const double* h_s,
                                           int d_s, double beta, double* out) {
  if (!rho || !h_star || !h_s || !out || d_s < 1 || d_s > 64 || !(beta > 0) || !std::isfinite(beta)) {
    set_error("rdm_energy_deviation: need non-NULL arrays, 1 <= d_s <= 64 and finite beta > 0");
    return RDM_EINVAL;
  }
  std::vector<double> hs, w(d_s), vt((size_t)d_s * d_s);
  if (!symmetrised(h_s, d_s, hs)) {
    set_error("rdm_energy_deviation: h_s has non-finite entries");
    return RDM_ENUMERIC;
  }
  if (!rdm::sym_eig(d_s, hs.data(), w.data(), vt.data())) {
    set_error("rdm_energy_deviation: eigensolver did not converge");
    return RDM_ENUMERIC;
  }
  // tr(H_s rho_s) = sum_j w_j e^{-beta (w_j - w_0)} / sum_j e^{-beta (w_j - w_0)}
  double z = 0.0, e_s = 0.0;
  for (int j = 0; j < d_s; ++j) {
    const double f = std::exp(-beta * (w[j] - w[0]));
    z += f;
    e_s += w[j] * f;
  }
  // tr(H* rho*) with both symmetrised
  double e_star = 0.0;
  for (int r = 0; r < d_s; ++r)
    for (int c = 0; c < d_s; ++c)
      e_star += 0.25 * (h_star[r * d_s + c] + h_star[c * d_s + r]) * (rho[c * d_s + r] + rho[r * d_s + c]);
  if (!std::isfinite(e_star)) {
    set_error("rdm_energy_deviation: h_star or rho has non-finite entries");
    return RDM_ENUMERIC;
  }
  *out = e_star - e_s / z;
  return RDM_OK;
}

extern "C" rdm_status rdm_entropy(const double* rho, int d_s, double* s_out) {
  if (!rho || !s_out || d_s < 1 || d_s > 64) {
    set_error("rdm_entropy: need rho, s_out and 1 <= d_s <= 64");
    return RDM_EINVAL;
  }
  std::vector<double> a, w(d_s);
  if (!symmetrised(rho, d_s, a)) {
    set_error("rdm_entropy: rho has non-finite entries");
    return RDM_ENUMERIC;
  }
  if (!rdm::sym_eig(d_s, a.data(), w.data(), nullptr)) {
    set_error("rdm_entropy: eigensolver did not converge");
    return RDM_ENUMERIC;
  }
  double s = 0.0;
  for (int j = 0; j < d_s; ++j)
    if (w[j] > 0) s -= w[j] * std::log(w[j]);
  *s_out = s;
  return RDM_OK;
}
