// Partially pivoted adaptive cross approximation of a coupling matrix
// (dfdm_aca; Sect. 2.7, closing remark: A_{c,t x s} ~ U V^* with k columns).
// Host code, a set-up step: it reads one row and one column of A per step.
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "dfdm_internal.cuh"

namespace dfdm {
namespace {

using cplx = std::complex<double>;

// A ~ sum_k u_k v_k^T.  Step k: the residual of row i_k; its largest entry
// (column j_k) is the pivot, v_k = residual row / pivot; u_k = residual of
// column j_k; ||S_k||_F^2 grows by |u_k|^2 |v_k|^2 + 2 Re sum_{l<k}
// (u_l^H u_k)(v_l^H v_k); stop once |u_k| |v_k| <= tol ||S_k||_F (the k-th
// term kept) or at max_rank; the next row is the largest |u_k| among rows
// not used yet.  A row whose residual is zero is marked used and the first
// unused row taken instead.
int aca_partial(const cplx *a, int m, int n, double tol, int max_rank, std::vector<cplx> &us,
                std::vector<cplx> &vs) {
  us.clear();
  vs.clear();
  std::vector<char> used(m, 0);
  std::vector<cplx> row(n), col(m);
  double fro2 = 0.0;
  int i = 0, k = 0, nused = 0;
  while (k < max_rank) {
    for (int j = 0; j < n; ++j) row[j] = a[(size_t)i * n + j];
    for (int l = 0; l < k; ++l) {
      const cplx ul = us[(size_t)l * m + i];
      for (int j = 0; j < n; ++j) row[j] -= ul * vs[(size_t)l * n + j];
    }
    if (!used[i]) {
      used[i] = 1;
      ++nused;
    }
    int jp = 0;
    double best = -1.0;
    for (int j = 0; j < n; ++j) {
      const double r = std::abs(row[j]);
      if (r > best) {
        best = r;
        jp = j;
      }
    }
    if (best == 0.0) {
      if (nused == m) break;
      i = 0;
      while (used[i]) ++i;
      continue;
    }
    const cplx piv = row[jp];
    for (int j = 0; j < n; ++j) row[j] /= piv;
    for (int r = 0; r < m; ++r) col[r] = a[(size_t)r * n + jp];
    for (int l = 0; l < k; ++l) {
      const cplx vl = vs[(size_t)l * n + jp];
      for (int r = 0; r < m; ++r) col[r] -= vl * us[(size_t)l * m + r];
    }
    double nu2 = 0.0, nv2 = 0.0;
    for (int r = 0; r < m; ++r) nu2 += std::norm(col[r]);
    for (int j = 0; j < n; ++j) nv2 += std::norm(row[j]);
    cplx cross = 0.0;
    for (int l = 0; l < k; ++l) {
      cplx du = 0.0, dv = 0.0;
      for (int r = 0; r < m; ++r) du += std::conj(us[(size_t)l * m + r]) * col[r];
      for (int j = 0; j < n; ++j) dv += std::conj(vs[(size_t)l * n + j]) * row[j];
      cross += du * dv;
    }
    fro2 += nu2 * nv2 + 2.0 * cross.real();
    us.insert(us.end(), col.begin(), col.end());
    vs.insert(vs.end(), row.begin(), row.end());
    ++k;
    if (std::sqrt(nu2 * nv2) <= tol * std::sqrt(std::max(fro2, 0.0))) break;
    if (nused == m) break;
    double bu = -1.0;
    for (int r = 0; r < m; ++r) {
      if (used[r]) continue;
      const double ar = std::abs(col[r]);
      if (ar > bu) {
        bu = ar;
        i = r;
      }
    }
  }
  return k;
}

}  // namespace
}  // namespace dfdm

extern "C" dfdm_status dfdm_aca(const void *a, int m, int n, double tol, int max_rank, void *u, void *v,
                                int *rank) {
  if (!a || !rank || m < 1 || n < 1 || !(tol >= 0.0) || max_rank < 0 || (max_rank > 0 && (!u || !v))) {
    dfdm::set_error("dfdm_aca: invalid argument");
    return DFDM_ERR_INVALID_ARG;
  }
  try {
    const int kmax = std::min(max_rank, std::min(m, n));
    std::vector<std::complex<double>> us, vs;
    const int k = dfdm::aca_partial(static_cast<const std::complex<double> *>(a), m, n, tol, kmax, us, vs);
    auto *uo = static_cast<std::complex<double> *>(u);
    auto *vo = static_cast<std::complex<double> *>(v);
    // U (m x max_rank, row-major): column l = u_l; V (n x max_rank): column l = conj(v_l)
    for (int r = 0; r < m && kmax > 0; ++r)
      for (int l = 0; l < max_rank; ++l) uo[(size_t)r * max_rank + l] = l < k ? us[(size_t)l * m + r] : 0.0;
    for (int j = 0; j < n && kmax > 0; ++j)
      for (int l = 0; l < max_rank; ++l)
        vo[(size_t)j * max_rank + l] = l < k ? std::conj(vs[(size_t)l * n + j]) : 0.0;
    *rank = k;
    return DFDM_OK;
  } catch (const std::bad_alloc &) {
    dfdm::set_error("dfdm_aca: host allocation failed");
    return DFDM_ERR_OOM;
  }
}
