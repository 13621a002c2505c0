// P1 finite-element stiffness and row-sum lumped mass (Sec. 2.1, Eq. sd_sys).
//
// K_ij = sum_T int_T D grad(phi_j) . grad(phi_i), M_ii = sum_{T ∋ i} |T| / (dim+1).
// Row-wise assembly: node -> cell incidence by counting sort, the sorted
// unique neighbour set of every row, then each row accumulates the
// contributions of its incident cells in ascending cell order (deterministic
// and free of write conflicts, so rows are processed in parallel).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "emrkc.h"

namespace {

// Gradients of the dim+1 barycentric functions of a simplex and its volume.
// J has the edge vectors x_k - x_0 as columns; grad(phi_k) (k >= 1) is row
// k-1 of J^{-1}, grad(phi_0) = -sum_k grad(phi_k).
bool simplex_gradients(int dim, const double* X, double* G, double* vol) {
  if (dim == 1) {
    const double h = X[1] - X[0];
    if (h == 0.0) return false;
    G[1] = 1.0 / h;
    G[0] = -G[1];
    *vol = std::fabs(h);
    return true;
  }
  if (dim == 2) {
    const double a = X[2] - X[0], b = X[4] - X[0];  // first row of J: x-components
    const double c = X[3] - X[1], d = X[5] - X[1];  // second row: y-components
    const double det = a * d - b * c;
    if (det == 0.0) return false;
    // J^{-1} = [d -b; -c a] / det
    G[2 + 0] = d / det;
    G[2 + 1] = -b / det;
    G[4 + 0] = -c / det;
    G[4 + 1] = a / det;
    G[0] = -(G[2] + G[4]);
    G[1] = -(G[3] + G[5]);
    *vol = std::fabs(det) / 2.0;
    return true;
  }
  // dim == 3: J columns e_k = X_k - X_0; J^{-1} rows are (e_2 x e_3, e_3 x e_1, e_1 x e_2) / det
  double e[3][3];
  for (int k = 0; k < 3; ++k)
    for (int c = 0; c < 3; ++c) e[k][c] = X[(k + 1) * 3 + c] - X[c];
  auto cross = [](const double* u, const double* v, double* w) {
    w[0] = u[1] * v[2] - u[2] * v[1];
    w[1] = u[2] * v[0] - u[0] * v[2];
    w[2] = u[0] * v[1] - u[1] * v[0];
  };
  double r[3][3];
  cross(e[1], e[2], r[0]);
  cross(e[2], e[0], r[1]);
  cross(e[0], e[1], r[2]);
  const double det = e[0][0] * r[0][0] + e[0][1] * r[0][1] + e[0][2] * r[0][2];
  if (det == 0.0) return false;
  for (int k = 0; k < 3; ++k)
    for (int c = 0; c < 3; ++c) G[(k + 1) * 3 + c] = r[k][c] / det;
  for (int c = 0; c < 3; ++c) G[c] = -(G[3 + c] + G[6 + c] + G[9 + c]);
  *vol = std::fabs(det) / 6.0;
  return true;
}

}  // namespace

extern "C" {

void emrkc_free_matrix(emrkc_owned_matrix* m) {
  if (!m) return;
  std::free(m->row_ptr);
  std::free(m->col);
  std::free(m->K);
  std::free(m->lumped_mass);
  std::memset(m, 0, sizeof(*m));
}

int emrkc_assemble_p1(int dim, int64_t n_nodes, const double* xyz, int64_t n_cells, const int64_t* cells,
                      const double* D, emrkc_owned_matrix* out) {
  if (!out) return EMRKC_ERR_ARG;
  std::memset(out, 0, sizeof(*out));
  if (dim < 1 || dim > 3 || n_nodes <= 0 || n_cells < 0 || !xyz || (n_cells > 0 && (!cells || !D)))
    return EMRKC_ERR_ARG;
  if (n_nodes > (int64_t)INT32_MAX - 64) return EMRKC_ERR_ARG;
  const int nv = dim + 1;
  for (int64_t c = 0; c < n_cells * nv; ++c)
    if (cells[c] < 0 || cells[c] >= n_nodes) return EMRKC_ERR_ARG;

  // node -> incident cells (counting sort keeps ascending cell order)
  std::vector<int64_t> inc_ptr(n_nodes + 1, 0);
  for (int64_t c = 0; c < n_cells * nv; ++c) inc_ptr[cells[c] + 1]++;
  for (int64_t i = 0; i < n_nodes; ++i) inc_ptr[i + 1] += inc_ptr[i];
  std::vector<int64_t> inc(inc_ptr[n_nodes]);
  {
    std::vector<int64_t> fill(inc_ptr.begin(), inc_ptr.end() - 1);
    for (int64_t c = 0; c < n_cells; ++c)
      for (int a = 0; a < nv; ++a) inc[fill[cells[c * nv + a]]++] = c;
  }

  // row patterns
  std::vector<int64_t> row_ptr(n_nodes + 1, 0);
  bool bad = false;
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t i = 0; i < n_nodes; ++i) {
    std::vector<int64_t> nb;
    nb.reserve((inc_ptr[i + 1] - inc_ptr[i]) * nv);
    for (int64_t p = inc_ptr[i]; p < inc_ptr[i + 1]; ++p)
      for (int a = 0; a < nv; ++a) nb.push_back(cells[inc[p] * nv + a]);
    std::sort(nb.begin(), nb.end());
    row_ptr[i + 1] = std::unique(nb.begin(), nb.end()) - nb.begin();
  }
  for (int64_t i = 0; i < n_nodes; ++i) row_ptr[i + 1] += row_ptr[i];
  const int64_t nnz = row_ptr[n_nodes];
  int32_t* col = (int32_t*)std::malloc(std::max<int64_t>(nnz, 1) * sizeof(int32_t));
  double* K = (double*)std::calloc(std::max<int64_t>(nnz, 1), sizeof(double));
  double* M = (double*)std::calloc(n_nodes, sizeof(double));
  int64_t* rp = (int64_t*)std::malloc((n_nodes + 1) * sizeof(int64_t));
  if (!col || !K || !M || !rp) {
    std::free(col);
    std::free(K);
    std::free(M);
    std::free(rp);
    return EMRKC_ERR_OOM;
  }
  std::memcpy(rp, row_ptr.data(), (n_nodes + 1) * sizeof(int64_t));

#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t i = 0; i < n_nodes; ++i) {
    std::vector<int64_t> nb;
    for (int64_t p = inc_ptr[i]; p < inc_ptr[i + 1]; ++p)
      for (int a = 0; a < nv; ++a) nb.push_back(cells[inc[p] * nv + a]);
    std::sort(nb.begin(), nb.end());
    nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
    int32_t* rc = col + row_ptr[i];
    double* rk = K + row_ptr[i];
    for (size_t k = 0; k < nb.size(); ++k) rc[k] = (int32_t)nb[k];
    double X[12], G[12], vol;
    double mass = 0.0;
    for (int64_t p = inc_ptr[i]; p < inc_ptr[i + 1]; ++p) {
      const int64_t c = inc[p];
      int li = -1;
      for (int a = 0; a < nv; ++a) {
        const int64_t node = cells[c * nv + a];
        if (node == i && li < 0) li = a;
        for (int d = 0; d < dim; ++d) X[a * dim + d] = xyz[node * dim + d];
      }
      if (!simplex_gradients(dim, X, G, &vol)) {
        bad = true;
        continue;
      }
      const double* Dc = D + c * dim * dim;
      // D grad(phi_li)
      double Dg[3] = {0, 0, 0};
      for (int r = 0; r < dim; ++r)
        for (int q = 0; q < dim; ++q) Dg[r] += Dc[r * dim + q] * G[li * dim + q];
      for (int b = 0; b < nv; ++b) {
        double dot = 0.0;
        for (int r = 0; r < dim; ++r) dot += G[b * dim + r] * Dg[r];
        const int64_t node = cells[c * nv + b];
        const int32_t* pos = std::lower_bound(rc, rc + nb.size(), (int32_t)node);
        rk[pos - rc] += vol * dot;
      }
      mass += vol / (double)nv;
    }
    M[i] = mass;
  }
  if (bad) {
    std::free(col);
    std::free(K);
    std::free(M);
    std::free(rp);
    return EMRKC_ERR_ARG;
  }
  out->n = n_nodes;
  out->nnz = nnz;
  out->row_ptr = rp;
  out->col = col;
  out->K = K;
  out->lumped_mass = M;
  return EMRKC_OK;
}

}  // extern "C"
