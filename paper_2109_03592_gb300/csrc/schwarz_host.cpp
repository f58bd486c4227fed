// Host-side set-up of the local solves of the overlapping Schwarz
// preconditioner (Sec. 2, Eq. 6), in fast-diagonalisation form.
//
// Each subdomain is one element with all its GLL nodes (the overlap is the
// shared nodes).  Its local problem is approximated by the separable
//   h1 (B_t (x) B_s (x) K_r + B_t (x) K_s (x) B_r + K_t (x) B_s (x) B_r) + h2 B_t (x) B_s (x) B_r
// from 1D operators per reference direction: with the element's mean length
// l along that direction, K = (2/l) D^T W D and B = (l/2) W on its n GLL
// points; at an end shared with a neighbour of mean length l' normal to the
// shared face, K[end][end] += (2/l') (D^T W D)[N][N] and B[end][end] +=
// (l'/2) w_N; an end on a Dirichlet face is decoupled (off-diagonal entries of
// K removed).  The generalised eigenproblem K S = B S diag(lam), S^T B S = I,
// is solved as the symmetric one for B^{-1/2} K B^{-1/2} (B is diagonal) by
// cyclic Jacobi rotations.  On an axis-aligned box these local operators are
// the exact principal submatrices of the assembled operator.  Two element
// faces are neighbours when they have the same four vertices.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "schwarz.h"
#include "sem_internal.h"

namespace sem {
namespace {

// Eigen-decomposition of the symmetric n x n matrix A (row-major, destroyed):
// A = V diag(lam) V^T, V orthogonal (columns), lam ascending.
void jacobi_eigen(int n, std::vector<double>& A, std::vector<double>& V, std::vector<double>& lam) {
  V.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int p = 0; p < n; ++p) {
      diag += A[p * n + p] * A[p * n + p];
      for (int q = p + 1; q < n; ++q) off += A[p * n + q] * A[p * n + q];
    }
    if (off <= 1e-32 * diag) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[p * n + q];
        if (apq == 0.0) continue;
        // the rotation that zeroes A[p][q]: the 2-by-2 symmetric Schur decomposition of
        // the classical Jacobi method (Golub & Van Loan, Matrix Computations)
        const double tau = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < n; ++k) {  // A <- A J (columns p, q)
          const double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // A <- J^T A (rows p, q)
          const double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {  // V <- V J
          const double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return A[a * n + a] < A[b * n + b]; });
  std::vector<double> V2(n * n);
  lam.assign(n, 0.0);
  for (int c = 0; c < n; ++c) {
    lam[c] = A[ord[c] * n + ord[c]];
    for (int k = 0; k < n; ++k) V2[k * n + c] = V[k * n + ord[c]];
  }
  V.swap(V2);
}

// S [n][n] (row-major, columns the eigenvectors) and lam [n]; l_lo / l_hi <= 0: no neighbour.
void fdm_1d(int N, const std::vector<double>& w, const std::vector<double>& Kref, double l, double l_lo, double l_hi,
            bool d_lo, bool d_hi, double* S, double* lam) {
  const int n = N + 1;
  std::vector<double> K(n * n), B(n);
  for (int q = 0; q < n * n; ++q) K[q] = (2.0 / l) * Kref[q];
  for (int i = 0; i < n; ++i) B[i] = 0.5 * l * w[i];
  const int ends[2] = {0, N};
  const double ln[2] = {l_lo, l_hi};
  const bool dir[2] = {d_lo, d_hi};
  for (int t = 0; t < 2; ++t) {
    const int e = ends[t];
    if (dir[t]) {
      for (int k = 0; k < n; ++k)
        if (k != e) K[e * n + k] = K[k * n + e] = 0.0;
    } else if (ln[t] > 0.0) {
      K[e * n + e] += (2.0 / ln[t]) * Kref[N * n + N];
      B[e] += 0.5 * ln[t] * w[N];
    }
  }
  std::vector<double> C(n * n), V, ev;
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) C[i * n + k] = K[i * n + k] / std::sqrt(B[i] * B[k]);
  jacobi_eigen(n, C, V, ev);
  for (int i = 0; i < n; ++i) {
    const double sc = 1.0 / std::sqrt(B[i]);
    for (int c = 0; c < n; ++c) S[i * n + c] = sc * V[i * n + c];
  }
  for (int c = 0; c < n; ++c) lam[c] = ev[c];
}

void reference_stiffness(int N, std::vector<double>& w, std::vector<double>& Kref) {
  const int n = N + 1;
  std::vector<double> xi, D;
  gll(N, xi, w, D);
  Kref.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      double s = 0.0;
      for (int q = 0; q < n; ++q) s += D[q * n + i] * w[q] * D[q * n + k];
      Kref[i * n + k] = s;
    }
}

}  // namespace
}  // namespace sem

namespace sem {

sem_status fdm_tables(int64_t E, int N, const int64_t* glo, const double* xyz, const uint8_t* dirichlet_face,
                      FdmTables& out) {
  const int n = N + 1, n2 = n * n, n3 = n2 * n;
  // mean element lengths along r, s, t: the mean over the n^2 GLL lines of the distance between their ends
  std::vector<double> L(3 * E);
  for (int64_t e = 0; e < E; ++e) {
    const double* x = xyz + e * 3 * n3;
    for (int a = 0; a < 3; ++a) {
      const int stride = a == 0 ? 1 : (a == 1 ? n : n2);
      double sum = 0.0;
      for (int u = 0; u < n; ++u)
        for (int v = 0; v < n; ++v) {
          // the line's start: index 0 along a, (u, v) along the other two
          int start;
          if (a == 0) start = n * u + n2 * v;
          else if (a == 1) start = u + n2 * v;
          else start = u + n * v;
          double d2 = 0.0;
          for (int c = 0; c < 3; ++c) {
            const double dx = x[c * n3 + start + N * stride] - x[c * n3 + start];
            d2 += dx * dx;
          }
          sum += std::sqrt(d2);
        }
      L[3 * e + a] = sum / (double)n2;
    }
  }
  // face neighbours: two element faces are one face when they have the same
  // four vertices (the sorted global ids of their corner nodes), whatever the
  // orientation of the two elements
  auto corner = [&](int a, int end, int u, int v) {
    const int cu = u ? N : 0, cv = v ? N : 0;
    return a == 0 ? end + n * cu + n2 * cv : (a == 1 ? cu + n * end + n2 * cv : cu + n * cv + n2 * end);
  };
  std::map<std::array<int64_t, 4>, std::vector<std::pair<int64_t, int>>> owner;
  for (int64_t e = 0; e < E; ++e)
    for (int f = 0; f < 6; ++f) {
      const int a = f / 2, end = (f % 2 == 0) ? 0 : N;
      std::array<int64_t, 4> key;
      for (int q = 0; q < 4; ++q) key[q] = glo[e * n3 + corner(a, end, q & 1, q >> 1)];
      std::sort(key.begin(), key.end());
      owner[key].push_back({e, f});
    }
  std::vector<double> nbl(6 * E, -1.0);
  for (const auto& kv : owner) {
    if (kv.second.size() != 2) continue;
    const auto a = kv.second[0], b = kv.second[1];
    nbl[6 * a.first + a.second] = L[3 * b.first + b.second / 2];
    nbl[6 * b.first + b.second] = L[3 * a.first + a.second / 2];
  }
  // 1D problems, each distinct (l, l_lo, l_hi, Dirichlet ends) solved once
  std::vector<double> w, Kref;
  reference_stiffness(N, w, Kref);
  using Key = std::tuple<double, double, double, int>;
  std::map<Key, int32_t> seen;  // key -> row of the distinct tables
  out.S.clear();
  out.lam.clear();
  out.sidx.assign(3 * E, 0);
  for (int64_t e = 0; e < E; ++e)
    for (int a = 0; a < 3; ++a) {
      const bool dlo = dirichlet_face[6 * e + 2 * a] != 0, dhi = dirichlet_face[6 * e + 2 * a + 1] != 0;
      const double llo = dlo ? 0.0 : nbl[6 * e + 2 * a], lhi = dhi ? 0.0 : nbl[6 * e + 2 * a + 1];
      const Key key{L[3 * e + a], llo, lhi, (dlo ? 1 : 0) | (dhi ? 2 : 0)};
      auto it = seen.find(key);
      if (it == seen.end()) {
        const int32_t row = (int32_t)seen.size();
        out.S.resize((size_t)(row + 1) * n2);
        out.lam.resize((size_t)(row + 1) * n);
        fdm_1d(N, w, Kref, L[3 * e + a], llo, lhi, dlo, dhi, out.S.data() + (size_t)row * n2,
               out.lam.data() + (size_t)row * n);
        it = seen.emplace(key, row).first;
      }
      out.sidx[3 * e + a] = it->second;
    }
  out.nd = (int64_t)seen.size();
  return SEM_OK;
}

}  // namespace sem

using namespace sem;

extern "C" {

sem_status sem_schwarz_fdm_1d(int N, double l, double l_lo, double l_hi, int dir_lo, int dir_hi, double* S_host,
                              double* lam_host) {
  if (N < 1 || N > kMaxN || !(l > 0.0) || !S_host || !lam_host) {
    set_error("sem_schwarz_fdm_1d: need N in [1, 11], l > 0 and output arrays");
    return SEM_ERR_INVALID;
  }
  std::vector<double> w, Kref;
  reference_stiffness(N, w, Kref);
  fdm_1d(N, w, Kref, l, l_lo, l_hi, dir_lo != 0, dir_hi != 0, S_host, lam_host);
  return SEM_OK;
}

sem_status sem_schwarz_setup_host(int64_t E, int N, const int64_t* glo, const double* xyz,
                                  const uint8_t* dirichlet_face, double* S_host, double* lam_host,
                                  int64_t* n_distinct) {
  SEM_TRACE("sem_schwarz_setup_host");
  if (E < 1 || N < 1 || N > kMaxN || !glo || !xyz || !dirichlet_face || !S_host || !lam_host) {
    set_error("sem_schwarz_setup_host: need E >= 1, N in [1, 11] and non-null arrays");
    return SEM_ERR_INVALID;
  }
  const int n = N + 1, n2 = n * n;
  FdmTables t;
  sem_status st = fdm_tables(E, N, glo, xyz, dirichlet_face, t);
  if (st != SEM_OK) return st;
  for (int64_t slot = 0; slot < 3 * E; ++slot) {
    const int32_t row = t.sidx[slot];
    std::memcpy(S_host + slot * n2, t.S.data() + (size_t)row * n2, sizeof(double) * n2);
    std::memcpy(lam_host + slot * n, t.lam.data() + (size_t)row * n, sizeof(double) * n);
  }
  if (n_distinct) *n_distinct = t.nd;
  return SEM_OK;
}

}  // extern "C"
