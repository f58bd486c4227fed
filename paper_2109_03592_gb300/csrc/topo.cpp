// Host-side mesh construction: GLL points, the built-in box/pipe topologies,
// the topological first-touch global numbering and the gather-scatter plan.
//
// Sec. 2 of the paper splits the SEM operator into local tensor-product work
// and a global "exchange of element face values" over GLL nodes shared by
// neighbouring elements.  This file builds the index structures for that
// exchange from element corner vertex ids alone:
//   * a GLL node on an element vertex is keyed by the vertex id;
//   * a node inside an edge by the edge (unordered vertex pair) and its
//     distance from the edge's lower-id vertex;
//   * a node inside a face by the face (its 4 vertex ids) and its
//     coordinates in the face's canonical frame (origin at the lowest-id
//     corner, first axis toward the lower-id neighbouring corner);
//   * an element-interior node is unique to its element.
// Global ids are then given in order of first appearance over local points
// in ascending local index l = i + n (j + n (k + n e)).
#include <algorithm>
#include <array>
#include <cmath>
#include <numeric>

#include "sem_internal.h"

namespace sem {

// ---- GLL -------------------------------------------------------------------

// Legendre P_N(x) and P_{N-1}(x) by the three-term recurrence.
static void legendre_pair(int N, double x, double& pN, double& pNm1) {
  double p0 = 1.0, p1 = x;
  if (N == 0) { pN = 1.0; pNm1 = 0.0; return; }
  for (int k = 1; k < N; ++k) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  pN = p1;
  pNm1 = p0;
}

void gll(int N, std::vector<double>& xi, std::vector<double>& w, std::vector<double>& D) {
  const int n = N + 1;
  xi.assign(n, 0.0);
  w.assign(n, 0.0);
  D.assign(n * n, 0.0);
  xi[0] = -1.0;
  xi[N] = 1.0;
  // Interior nodes: roots of P_N'.  Newton on P_N' with
  //   (1 - x^2) P_N'  = N (P_{N-1} - x P_N)
  //   (1 - x^2) P_N'' = 2 x P_N' - N (N+1) P_N      (Legendre's equation)
  for (int i = 1; i < N; ++i) {
    double x = -std::cos(M_PI * i / N);
    for (int it = 0; it < 100; ++it) {
      double pN, pNm1;
      legendre_pair(N, x, pN, pNm1);
      const double s = 1.0 - x * x;
      const double d1 = N * (pNm1 - x * pN) / s;
      const double d2 = (2.0 * x * d1 - N * (N + 1.0) * pN) / s;
      const double dx = d1 / d2;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    xi[i] = x;
  }
  std::sort(xi.begin(), xi.end());
  for (int i = 0; i < n; ++i) {
    double pN, pNm1;
    legendre_pair(N, xi[i], pN, pNm1);
    w[i] = 2.0 / (N * (N + 1.0) * pN * pN);
  }
  // D by barycentric Lagrange differentiation: lambda_j = 1 / prod_{k!=j}(x_j - x_k),
  // D_ij = (lambda_j / lambda_i) / (x_i - x_j) for i != j, D_ii = -sum_{j!=i} D_ij.
  std::vector<double> lam(n, 1.0);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k)
      if (k != j) lam[j] /= (xi[j] - xi[k]);
  for (int i = 0; i < n; ++i) {
    double diag = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      const double v = (lam[j] / lam[i]) / (xi[i] - xi[j]);
      D[i * n + j] = v;
      diag -= v;
    }
    D[i * n + i] = diag;
  }
}

// ---- built-in generators ----------------------------------------------------

static sem_status check_desc(const sem_mesh_desc& d) {
  if (d.N < 1 || d.N > kMaxN) { set_error("N must be in [1, 11]"); return SEM_ERR_INVALID; }
  if (d.kind == SEM_MESH_BOX) {
    if (d.nx < 1 || d.ny < 1 || d.nz < 1 || !(d.lx > 0) || !(d.ly > 0) || !(d.lz > 0)) {
      set_error("box: need nx, ny, nz >= 1 and positive lengths");
      return SEM_ERR_INVALID;
    }
  } else if (d.kind == SEM_MESH_PIPE) {
    if (d.nc < 1 || d.nr < 1 || d.nzp < 1 || !(d.R > 0) || !(d.L > 0) || !(d.beta > 0) ||
        !(d.a > 0) || !(d.a < d.R / std::sqrt(2.0))) {
      set_error("pipe: need nc, nr, nzp >= 1, R, L, beta > 0 and 0 < a < R/sqrt(2)");
      return SEM_ERR_INVALID;
    }
    if (d.periodic_z && d.nzp < 3) {
      set_error("pipe: a periodic pipe needs nzp >= 3 (vertex ids must identify every edge)");
      return SEM_ERR_INVALID;
    }
  } else if (d.kind == SEM_MESH_EXPLICIT) {
    if (d.E < 1 || !d.xyz || !d.vert || !d.dirichlet_face) {
      set_error("explicit mesh: need E >= 1 and xyz, vert, dirichlet_face");
      return SEM_ERR_INVALID;
    }
  } else {
    set_error("unknown mesh kind");
    return SEM_ERR_INVALID;
  }
  return SEM_OK;
}

// 2D vertex id of the pipe cross-section: square vertex (ix, iy), or a ring
// vertex at radial level L >= 1 and tangential index T of block q.
static int64_t pipe_v2d(int nc, int q, int level, int T) {
  if (level == 0) {
    int ix, iy;
    switch (q) {
      case 0: ix = nc; iy = T; break;
      case 1: ix = nc - T; iy = nc; break;
      case 2: ix = 0; iy = nc - T; break;
      default: ix = T; iy = 0; break;
    }
    return (int64_t)iy * (nc + 1) + ix;
  }
  const int64_t ring = 4LL * nc;
  return (int64_t)(nc + 1) * (nc + 1) + (int64_t)(level - 1) * ring + ((int64_t)q * nc + T) % ring;
}

sem_status generator_vertices(const sem_mesh_desc& d, std::vector<int64_t>& vert, int64_t& E) {
  sem_status st = check_desc(d);
  if (st != SEM_OK) return st;
  if (d.kind == SEM_MESH_BOX) {
    E = (int64_t)d.nx * d.ny * d.nz;
    vert.resize(8 * E);
    auto vid = [&](int64_t ix, int64_t iy, int64_t iz) { return ix + (d.nx + 1) * (iy + (int64_t)(d.ny + 1) * iz); };
    for (int64_t e = 0; e < E; ++e) {
      const int64_t ex = e % d.nx, ey = (e / d.nx) % d.ny, ez = e / ((int64_t)d.nx * d.ny);
      for (int c = 0; c < 8; ++c) vert[8 * e + c] = vid(ex + (c & 1), ey + ((c >> 1) & 1), ez + (c >> 2));
    }
    return SEM_OK;
  }
  if (d.kind == SEM_MESH_PIPE) {
    const int nc = d.nc, nr = d.nr;
    const int64_t n2d = (int64_t)nc * (nc + 4 * nr);
    const int64_t nv2 = (int64_t)(nc + 1) * (nc + 1) + 4LL * nc * nr;
    E = n2d * d.nzp;
    vert.resize(8 * E);
    std::vector<int64_t> c2(4 * n2d);  // [e2d][a + 2b] 2D corner ids
    for (int ey = 0; ey < nc; ++ey)
      for (int ex = 0; ex < nc; ++ex)
        for (int c = 0; c < 4; ++c)
          c2[4 * (ey * nc + ex) + c] = (int64_t)(ey + (c >> 1)) * (nc + 1) + ex + (c & 1);
    for (int q = 0; q < 4; ++q)
      for (int r = 0; r < nr; ++r)
        for (int m = 0; m < nc; ++m) {
          const int64_t e2 = (int64_t)nc * nc + (int64_t)q * nc * nr + (int64_t)r * nc + m;
          for (int c = 0; c < 4; ++c) c2[4 * e2 + c] = pipe_v2d(nc, q, r + (c & 1), m + (c >> 1));
        }
    for (int64_t e = 0; e < E; ++e) {
      const int64_t layer = e / n2d, e2 = e % n2d;
      for (int c = 0; c < 8; ++c) {
        int64_t lz = layer + (c >> 2);
        if (d.periodic_z) lz %= d.nzp;
        vert[8 * e + c] = lz * nv2 + c2[4 * e2 + (c & 3)];
      }
    }
    return SEM_OK;
  }
  E = d.E;
  vert.assign(d.vert, d.vert + 8 * E);
  return SEM_OK;
}

void generator_dirichlet(const sem_mesh_desc& d, int64_t E, std::vector<uint8_t>& dface) {
  dface.assign(6 * E, 0);
  if (d.kind == SEM_MESH_BOX) {
    for (int64_t e = 0; e < E; ++e) {
      const int64_t ex = e % d.nx, ey = (e / d.nx) % d.ny, ez = e / ((int64_t)d.nx * d.ny);
      dface[6 * e + 0] = ex == 0;
      dface[6 * e + 1] = ex == d.nx - 1;
      dface[6 * e + 2] = ey == 0;
      dface[6 * e + 3] = ey == d.ny - 1;
      dface[6 * e + 4] = ez == 0;
      dface[6 * e + 5] = ez == d.nz - 1;
    }
  } else if (d.kind == SEM_MESH_PIPE) {
    const int64_t n2d = (int64_t)d.nc * (d.nc + 4 * d.nr);
    for (int64_t e = 0; e < E; ++e) {
      const int64_t layer = e / n2d, e2 = e % n2d;
      if (e2 >= (int64_t)d.nc * d.nc) {
        const int64_t r = ((e2 - (int64_t)d.nc * d.nc) % ((int64_t)d.nc * d.nr)) / d.nc;
        dface[6 * e + 1] = r == d.nr - 1;
      }
      if (!d.periodic_z) {
        dface[6 * e + 4] = layer == 0;
        dface[6 * e + 5] = layer == d.nzp - 1;
      }
    }
  } else {
    for (int64_t q = 0; q < 6 * E; ++q) dface[q] = d.dirichlet_face[q] != 0;
  }
}

// ---- topological numbering --------------------------------------------------

namespace {

// Corner (start, end) of element edge `le` (0..11): 4 edges along i, then j, then k.
inline void edge_corners(int le, int& c0, int& c1) {
  const int dir = le / 4, o = le % 4, b0 = o & 1, b1 = o >> 1;
  if (dir == 0) { c0 = 2 * b0 + 4 * b1; c1 = c0 + 1; }
  else if (dir == 1) { c0 = b0 + 4 * b1; c1 = c0 + 2; }
  else { c0 = b0 + 2 * b1; c1 = c0 + 4; }
}

// Corner of face f at face-local corner (pb, qb); the face-local axes are
// (j, k) for faces 0/1, (i, k) for 2/3 and (i, j) for 4/5.
inline int face_corner(int f, int pb, int qb) {
  const int dir = f / 2, side = f % 2;
  if (dir == 0) return side + 2 * pb + 4 * qb;
  if (dir == 1) return pb + 2 * side + 4 * qb;
  return pb + 2 * qb + 4 * side;
}

}  // namespace

sem_status build_numbering(int64_t E, int N, const int64_t* vert, Topology& t) {
  if (E < 1 || N < 1 || N > kMaxN) { set_error("numbering: bad E or N"); return SEM_ERR_INVALID; }
  const int n = N + 1, Nm = N - 1;
  const int64_t n3 = (int64_t)n * n * n;
  t.E = E;
  t.N = N;
  t.n_local = E * n3;

  // compact vertex ids
  std::vector<int64_t> vs(vert, vert + 8 * E);
  std::sort(vs.begin(), vs.end());
  vs.erase(std::unique(vs.begin(), vs.end()), vs.end());
  const int64_t NV = (int64_t)vs.size();
  if (NV >= (1LL << 31)) { set_error("numbering: too many vertices"); return SEM_ERR_INVALID; }
  std::vector<int64_t> cv(8 * E);
  for (int64_t q = 0; q < 8 * E; ++q) cv[q] = std::lower_bound(vs.begin(), vs.end(), vert[q]) - vs.begin();
  for (int64_t e = 0; e < E; ++e) {
    std::array<int64_t, 8> c;
    for (int q = 0; q < 8; ++q) c[q] = cv[8 * e + q];
    std::sort(c.begin(), c.end());
    if (std::adjacent_find(c.begin(), c.end()) != c.end()) {
      set_error("numbering: an element repeats a corner vertex id");
      return SEM_ERR_BAD_MESH;
    }
  }

  // edges: key = min * NV + max
  std::vector<std::pair<uint64_t, int64_t>> ek(12 * E);
  for (int64_t e = 0; e < E; ++e)
    for (int le = 0; le < 12; ++le) {
      int c0, c1;
      edge_corners(le, c0, c1);
      const uint64_t a = cv[8 * e + c0], b = cv[8 * e + c1];
      ek[12 * e + le] = {std::min(a, b) * (uint64_t)NV + std::max(a, b), 12 * e + le};
    }
  std::sort(ek.begin(), ek.end());
  std::vector<int64_t> edge_id(12 * E);
  int64_t NE = 0;
  for (size_t q = 0; q < ek.size(); ++q) {
    if (q > 0 && ek[q].first != ek[q - 1].first) ++NE;
    edge_id[ek[q].second] = NE;
  }
  ++NE;

  // faces: key = the 4 sorted vertex ids; a conforming face is shared by <= 2 elements
  std::vector<std::pair<std::array<int64_t, 4>, int64_t>> fk(6 * E);
  for (int64_t e = 0; e < E; ++e)
    for (int f = 0; f < 6; ++f) {
      std::array<int64_t, 4> k4;
      for (int c = 0; c < 4; ++c) k4[c] = cv[8 * e + face_corner(f, c & 1, c >> 1)];
      std::sort(k4.begin(), k4.end());
      fk[6 * e + f] = {k4, 6 * e + f};
    }
  std::sort(fk.begin(), fk.end());
  std::vector<int64_t> face_id(6 * E);
  int64_t NF = 0;
  int run = 0;
  for (size_t q = 0; q < fk.size(); ++q) {
    if (q > 0 && fk[q].first != fk[q - 1].first) { ++NF; run = 0; }
    if (++run > 2) { set_error("numbering: a face is shared by more than two elements"); return SEM_ERR_BAD_MESH; }
    face_id[fk[q].second] = NF;
  }
  ++NF;

  // canonical frame of every element face: origin corner (o1, o2), swap flag
  std::vector<uint8_t> fframe(6 * E);
  for (int64_t e = 0; e < E; ++e)
    for (int f = 0; f < 6; ++f) {
      int best = 0;
      int64_t bv = cv[8 * e + face_corner(f, 0, 0)];
      for (int c = 1; c < 4; ++c) {
        const int64_t v = cv[8 * e + face_corner(f, c & 1, c >> 1)];
        if (v < bv) { bv = v; best = c; }
      }
      const int o1 = best & 1, o2 = best >> 1;
      const int64_t vp = cv[8 * e + face_corner(f, 1 - o1, o2)];  // neighbour along p
      const int64_t vq = cv[8 * e + face_corner(f, o1, 1 - o2)];  // neighbour along q
      const int swap = vq < vp;
      fframe[6 * e + f] = (uint8_t)(o1 | (o2 << 1) | (swap << 2));
    }

  const int64_t base_e = NV, base_f = NV + NE * Nm, base_i = base_f + NF * Nm * Nm;
  const int64_t K = base_i + E * (int64_t)Nm * Nm * Nm;
  std::vector<int64_t> first(K, -1);
  t.glo.resize(t.n_local);
  int64_t next = 0;
  int64_t l = 0;
  for (int64_t e = 0; e < E; ++e) {
    const int64_t* c8 = &cv[8 * e];
    for (int k = 0; k < n; ++k) {
      const int bk = (k == 0 || k == N);
      for (int j = 0; j < n; ++j) {
        const int bj = (j == 0 || j == N);
        for (int i = 0; i < n; ++i, ++l) {
          const int bi = (i == 0 || i == N);
          const int nb = bi + bj + bk;
          int64_t key;
          if (nb == 3) {
            key = c8[(i == N) + 2 * (j == N) + 4 * (k == N)];
          } else if (nb == 2) {
            int dir, p, o;
            if (!bi) { dir = 0; p = i; o = (j == N) + 2 * (k == N); }
            else if (!bj) { dir = 1; p = j; o = (i == N) + 2 * (k == N); }
            else { dir = 2; p = k; o = (i == N) + 2 * (j == N); }
            const int le = 4 * dir + o;
            int c0, c1;
            edge_corners(le, c0, c1);
            const int cp = c8[c0] < c8[c1] ? p : N - p;
            key = base_e + edge_id[12 * e + le] * Nm + (cp - 1);
          } else if (nb == 1) {
            int f, p, q;
            if (bi) { f = (i == N); p = j; q = k; }
            else if (bj) { f = 2 + (j == N); p = i; q = k; }
            else { f = 4 + (k == N); p = i; q = j; }
            const uint8_t fr = fframe[6 * e + f];
            const int dp = (fr & 1) ? N - p : p, dq = (fr & 2) ? N - q : q;
            const int c1 = (fr & 4) ? dq : dp, c2 = (fr & 4) ? dp : dq;
            key = base_f + face_id[6 * e + f] * Nm * Nm + (c1 - 1) + (int64_t)Nm * (c2 - 1);
          } else {
            key = base_i + e * Nm * Nm * Nm + (i - 1) + (int64_t)Nm * ((j - 1) + (int64_t)Nm * (k - 1));
          }
          if (first[key] < 0) first[key] = next++;
          t.glo[l] = first[key];
        }
      }
    }
  }
  t.n_global = next;
  if (next != K) {
    set_error("numbering: some vertex/edge/face key was never touched (inconsistent topology)");
    return SEM_ERR_BAD_MESH;
  }
  return SEM_OK;
}

// ---- gather-scatter plan ----------------------------------------------------

sem_status build_gs_plan(const Topology& t, const uint8_t* dface, GsPlan& plan) {
  const int n = t.N + 1;
  const int64_t n3 = (int64_t)n * n * n;
  std::vector<int32_t> count(t.n_global, 0);
  for (int64_t l = 0; l < t.n_local; ++l) count[t.glo[l]]++;
  std::vector<uint8_t> dir(t.n_global, 0);
  for (int64_t e = 0; e < t.E; ++e)
    for (int f = 0; f < 6; ++f) {
      if (!dface[6 * e + f]) continue;
      const int d = f / 2, side = (f % 2) ? t.N : 0;
      for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
          int i, j, k;
          if (d == 0) { i = side; j = a; k = b; }
          else if (d == 1) { i = a; j = side; k = b; }
          else { i = a; j = b; k = side; }
          dir[t.glo[e * n3 + i + n * (j + n * k)]] = 1;
        }
    }
  plan.wm.resize(t.n_local);
  for (int64_t l = 0; l < t.n_local; ++l) {
    const int32_t m = count[t.glo[l]];
    if (m > 127) { set_error("gs plan: a node has more than 127 copies"); return SEM_ERR_BAD_MESH; }
    plan.wm[l] = (uint8_t)(m | (dir[t.glo[l]] ? 0x80 : 0));
  }
  // class of every node: 0..6 for m = 2..8, 7 for m > 8, 8 for a Dirichlet singleton, -1 none
  auto cls_of = [&](int64_t g) -> int {
    const int32_t m = count[g];
    if (m >= 2 && m <= 8) return m - 2;
    if (m > 8) return 7;
    return dir[g] ? 8 : -1;
  };
  int64_t entries[kGsClasses] = {0};
  for (int64_t g = 0; g < t.n_global; ++g) {
    const int c = cls_of(g);
    if (c < 0) continue;
    plan.cnt[c]++;
    entries[c] += count[g];
  }
  int64_t total = 0;
  for (int c = 0; c < kGsClasses; ++c) {
    plan.off[c] = total;
    total += (entries[c] + 3) / 4 * 4;
    plan.n_nodes += plan.cnt[c];
    plan.n_points += entries[c];
  }
  if (total >= (1LL << 31) - 1 || t.n_local >= (1LL << 31) - 1) {
    set_error("gs plan: more than 2^31 local points");
    return SEM_ERR_INVALID;
  }
  plan.idx.assign(total, 0);
  plan.gptr.assign(plan.cnt[7] + 1, 0);
  // position of each node's tuple, in ascending global id within its class
  std::vector<int64_t> pos(t.n_global, -1);
  int64_t fill[kGsClasses];
  for (int c = 0; c < kGsClasses; ++c) fill[c] = plan.off[c];
  int64_t gnode = 0;
  for (int64_t g = 0; g < t.n_global; ++g) {
    const int c = cls_of(g);
    if (c < 0) continue;
    pos[g] = fill[c];
    fill[c] += count[g];
    if (c == 7) {
      plan.gptr[gnode + 1] = plan.gptr[gnode] + count[g];
      ++gnode;
    }
  }
  // work units, window by window over the global ids, class by class inside
  {
    int64_t done[kGsClasses] = {0};  // nodes of each class with a global id below the window's end
    const int64_t win = kGsWindow;
    for (int64_t g0 = 0; g0 < t.n_global; g0 += win) {
      const int64_t g1 = std::min<int64_t>(t.n_global, g0 + win);
      int64_t upto[kGsClasses];
      for (int c = 0; c < kGsClasses; ++c) upto[c] = done[c];
      for (int64_t g = g0; g < g1; ++g) {
        const int c = cls_of(g);
        if (c >= 0) ++upto[c];
      }
      for (int c = 0; c < kGsClasses; ++c) {
        for (int64_t q = done[c]; q < upto[c]; q += kGsUnitNodes) {
          plan.units.push_back(c);
          plan.units.push_back((int32_t)q);
          plan.units.push_back((int32_t)std::min<int64_t>(kGsUnitNodes, upto[c] - q));
          plan.units.push_back(0);
        }
        done[c] = upto[c];
      }
    }
    // the units of each class tile its nodes exactly, in order (the kernel
    // indexes tuples by them without further checks)
    int64_t next[kGsClasses] = {0};
    for (size_t u = 0; u + 3 < plan.units.size(); u += 4) {
      const int c = plan.units[u];
      if (c < 0 || c >= kGsClasses || plan.units[u + 1] != next[c] || plan.units[u + 2] < 1 ||
          plan.units[u + 2] > kGsUnitNodes) {
        set_error("gs plan: inconsistent work units");
        return SEM_ERR_INVALID;
      }
      next[c] += plan.units[u + 2];
    }
    for (int c = 0; c < kGsClasses; ++c)
      if (next[c] != plan.cnt[c]) {
        set_error("gs plan: work units do not cover every node");
        return SEM_ERR_INVALID;
      }
  }
  // local points in ascending local index fill each tuple in ascending order
  std::vector<int32_t> seen(t.n_global, 0);
  for (int64_t l = 0; l < t.n_local; ++l) {
    const int64_t g = t.glo[l];
    if (pos[g] < 0) continue;
    int32_t v = (int32_t)l;
    if (seen[g] == 0 && dir[g]) v |= (int32_t)0x80000000u;
    plan.idx[pos[g] + seen[g]++] = v;
  }
  return SEM_OK;
}

}  // namespace sem
