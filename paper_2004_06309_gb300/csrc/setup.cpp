// Host setup (frequency-independent): dofs, element matrices, global and local
// operator pieces, overlapping decomposition with partition of unity, coarse
// interpolation and Galerkin coarse pieces.  Eq. (1)-(4) of the method.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "host.h"

namespace hz {

static const int kTetEdge[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
static const int kTriEdge[3][2] = {{0, 1}, {0, 2}, {1, 2}};
static const int kTetFace[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};

int64_t Dofs::edge_id(int64_t a, int64_t b) const {
  if (a > b) std::swap(a, b);
  const int64_t key = a * nv + b;
  auto it = std::lower_bound(edge_key.begin(), edge_key.end(), key);
  return (it != edge_key.end() && *it == key) ? int64_t(it - edge_key.begin()) : -1;
}

void Dofs::face_dofs(const int32_t* f, int64_t* out) const {
  for (int i = 0; i < 3; i++) out[i] = f[i];
  if (order == 2)
    for (int e = 0; e < 3; e++) out[3 + e] = nv + edge_id(f[kTriEdge[e][0]], f[kTriEdge[e][1]]);
}

int64_t Csr::find(int64_t r, int64_t c) const {
  const int32_t* b = col.data() + ptr[r];
  const int32_t* e = col.data() + ptr[r + 1];
  const int32_t* it = std::lower_bound(b, e, int32_t(c));
  return (it != e && *it == c) ? int64_t(it - col.data()) : -1;
}

// ---------------------------------------------------------------------------
// Reference element tables.
//
// Stiffness: each P2 basis derivative d phi_a / d lambda_p is affine in lambda,
// alpha + sum_q beta_q lambda_q, so int (d_p phi_a)(d_q phi_b) / |T| follows from
// int lambda_q / |T| = 1/4 and int lambda_q lambda_r / |T| = (1 + delta_qr) / 20.
// Mass: the classical tables |T|/420 (P2 tet), |T|/20 (1 + delta) (P1 tet),
// |F|/180 (P2 triangle), |F|/12 (1 + delta) (P1 triangle).
// ---------------------------------------------------------------------------
struct RefTables {
  double S[2][10][10][4][4];
  double M[2][10][10];
  double F[2][6][6];
  RefTables() {
    std::memset(this, 0, sizeof(*this));
    for (int ord = 1; ord <= 2; ord++) {
      const int o = ord - 1;
      const int nb = ord == 1 ? 4 : 10;
      double al[10][4], be[10][4][4];
      std::memset(al, 0, sizeof(al));
      std::memset(be, 0, sizeof(be));
      for (int a = 0; a < nb; a++) {
        for (int p = 0; p < 4; p++) {
          if (ord == 1) {
            al[a][p] = (a == p) ? 1.0 : 0.0;
          } else if (a < 4) {       // 2 l_a^2 - l_a  ->  d/dl_p = delta_ap (4 l_a - 1)
            if (a == p) { al[a][p] = -1.0; be[a][p][a] = 4.0; }
          } else {                  // 4 l_i l_j  ->  4 (delta_ip l_j + delta_jp l_i)
            const int i = kTetEdge[a - 4][0], j = kTetEdge[a - 4][1];
            if (p == i) be[a][p][j] += 4.0;
            if (p == j) be[a][p][i] += 4.0;
          }
        }
      }
      for (int a = 0; a < nb; a++)
        for (int b = 0; b < nb; b++)
          for (int p = 0; p < 4; p++)
            for (int q = 0; q < 4; q++) {
              double sa = 0, sb = 0, bb = 0;
              for (int r = 0; r < 4; r++) { sa += be[a][p][r]; sb += be[b][q][r]; }
              for (int r = 0; r < 4; r++)
                for (int t = 0; t < 4; t++) bb += be[a][p][r] * be[b][q][t] * (r == t ? 2.0 : 1.0) / 20.0;
              S[o][a][b][p][q] = al[a][p] * al[b][q] + (al[a][p] * sb + al[b][q] * sa) / 4.0 + bb;
            }
      if (ord == 1) {
        for (int a = 0; a < 4; a++)
          for (int b = 0; b < 4; b++) M[o][a][b] = (a == b ? 2.0 : 1.0) / 20.0;
        for (int a = 0; a < 3; a++)
          for (int b = 0; b < 3; b++) F[o][a][b] = (a == b ? 2.0 : 1.0) / 12.0;
      } else {
        for (int a = 0; a < 10; a++)
          for (int b = 0; b < 10; b++) {
            double v;
            if (a < 4 && b < 4) v = (a == b) ? 6 : 1;
            else if (a < 4 || b < 4) {
              const int vv = a < 4 ? a : b, e = (a < 4 ? b : a) - 4;
              v = (kTetEdge[e][0] == vv || kTetEdge[e][1] == vv) ? -4 : -6;
            } else {
              const int* ea = kTetEdge[a - 4];
              const int* eb = kTetEdge[b - 4];
              const bool share = ea[0] == eb[0] || ea[0] == eb[1] || ea[1] == eb[0] || ea[1] == eb[1];
              v = (a == b) ? 32 : (share ? 16 : 8);
            }
            M[o][a][b] = v / 420.0;
          }
        for (int a = 0; a < 6; a++)
          for (int b = 0; b < 6; b++) {
            double v;
            if (a < 3 && b < 3) v = (a == b) ? 6 : -1;
            else if (a < 3 || b < 3) {
              const int vv = a < 3 ? a : b, e = (a < 3 ? b : a) - 3;
              v = (kTriEdge[e][0] == vv || kTriEdge[e][1] == vv) ? 0 : -4;
            } else {
              v = (a == b) ? 32 : 16;
            }
            F[o][a][b] = v / 180.0;
          }
      }
    }
  }
};
static const RefTables& ref() {
  static RefTables t;
  return t;
}

// Volume and barycentric gradients of a tet: rows of J^{-1} are grad lambda_1..3,
// computed as cross products of J's columns over det J.
static double tet_grads(const double* xyz, const int32_t* t, double g[4][3]) {
  const double* x0 = xyz + 3 * int64_t(t[0]);
  double a[3], b[3], c[3];
  for (int i = 0; i < 3; i++) {
    a[i] = xyz[3 * int64_t(t[1]) + i] - x0[i];
    b[i] = xyz[3 * int64_t(t[2]) + i] - x0[i];
    c[i] = xyz[3 * int64_t(t[3]) + i] - x0[i];
  }
  const double bc[3] = {b[1] * c[2] - b[2] * c[1], b[2] * c[0] - b[0] * c[2], b[0] * c[1] - b[1] * c[0]};
  const double ca[3] = {c[1] * a[2] - c[2] * a[1], c[2] * a[0] - c[0] * a[2], c[0] * a[1] - c[1] * a[0]};
  const double ab[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
  const double det = a[0] * bc[0] + a[1] * bc[1] + a[2] * bc[2];
  for (int i = 0; i < 3; i++) {
    g[1][i] = bc[i] / det;
    g[2][i] = ca[i] / det;
    g[3][i] = ab[i] / det;
    g[0][i] = -(g[1][i] + g[2][i] + g[3][i]);
  }
  return std::fabs(det) / 6.0;
}

static double tri_area(const double* xyz, const int32_t* f) {
  double u[3], v[3];
  for (int i = 0; i < 3; i++) {
    u[i] = xyz[3 * int64_t(f[1]) + i] - xyz[3 * int64_t(f[0]) + i];
    v[i] = xyz[3 * int64_t(f[2]) + i] - xyz[3 * int64_t(f[0]) + i];
  }
  const double w[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
  return 0.5 * std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
}

// Element stiffness K_e and unit mass M_e (nb x nb, row-major).
static void element(const Mesh& m, int order, int64_t e, double* Ke, double* Me) {
  double g[4][3];
  const double vol = tet_grads(m.xyz.data(), m.tets.data() + 4 * e, g);
  double G[4][4];
  for (int p = 0; p < 4; p++)
    for (int q = 0; q < 4; q++) G[p][q] = g[p][0] * g[q][0] + g[p][1] * g[q][1] + g[p][2] * g[q][2];
  const int o = order - 1, nb = order == 1 ? 4 : 10;
  const RefTables& R = ref();
  for (int a = 0; a < nb; a++)
    for (int b = 0; b < nb; b++) {
      double s = 0;
      for (int p = 0; p < 4; p++)
        for (int q = 0; q < 4; q++) s += G[p][q] * R.S[o][a][b][p][q];
      Ke[a * nb + b] = vol * s;
      Me[a * nb + b] = vol * R.M[o][a][b];
    }
}

void eval_basis(int order, const double l[4], double* out) {
  if (order == 1) {
    for (int i = 0; i < 4; i++) out[i] = l[i];
    return;
  }
  for (int i = 0; i < 4; i++) out[i] = l[i] * (2.0 * l[i] - 1.0);
  for (int e = 0; e < 6; e++) out[4 + e] = 4.0 * l[kTetEdge[e][0]] * l[kTetEdge[e][1]];
}

static void barycentric(const double* xyz, const int32_t* t, const double* p, double l[4]) {
  double g[4][3];
  tet_grads(xyz, t, g);
  const double* x0 = xyz + 3 * int64_t(t[0]);
  double s = 0;
  for (int k = 1; k < 4; k++) {
    l[k] = g[k][0] * (p[0] - x0[0]) + g[k][1] * (p[1] - x0[1]) + g[k][2] * (p[2] - x0[2]);
    s += l[k];
  }
  l[0] = 1.0 - s;
}

// ---------------------------------------------------------------------------
void build_dofs(const Mesh& m, int order, Dofs& d) {
  d.order = order;
  d.nb = order == 1 ? 4 : 10;
  d.nbf = order == 1 ? 3 : 6;
  d.nv = m.nv;
  d.edge_key.clear();
  if (order == 2) {
    std::vector<int64_t> keys(size_t(m.ne) * 6);
    for (int64_t e = 0; e < m.ne; e++)
      for (int k = 0; k < 6; k++) {
        int64_t a = m.tets[4 * e + kTetEdge[k][0]], b = m.tets[4 * e + kTetEdge[k][1]];
        if (a > b) std::swap(a, b);
        keys[6 * e + k] = a * m.nv + b;
      }
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    d.edge_key.swap(keys);
  }
  d.n = m.nv + int64_t(d.edge_key.size());
  d.elem.resize(size_t(m.ne) * d.nb);
  for (int64_t e = 0; e < m.ne; e++) {
    for (int k = 0; k < 4; k++) d.elem[d.nb * e + k] = m.tets[4 * e + k];
    if (order == 2)
      for (int k = 0; k < 6; k++)
        d.elem[d.nb * e + 4 + k] = m.nv + d.edge_id(m.tets[4 * e + kTetEdge[k][0]], m.tets[4 * e + kTetEdge[k][1]]);
  }
  d.coord.resize(size_t(d.n) * 3);
  std::copy(m.xyz.begin(), m.xyz.end(), d.coord.begin());
  for (size_t k = 0; k < d.edge_key.size(); k++) {
    const int64_t a = d.edge_key[k] / m.nv, b = d.edge_key[k] % m.nv;
    for (int i = 0; i < 3; i++) d.coord[3 * (m.nv + k) + i] = 0.5 * (m.xyz[3 * a + i] + m.xyz[3 * b + i]);
  }
  d.is_dir.assign(d.n, 0);
  const int64_t nf = int64_t(m.tag.size());
  int64_t fd[6];
  for (int64_t f = 0; f < nf; f++)
    if (m.tag[f] == 0) {
      d.face_dofs(m.faces.data() + 3 * f, fd);
      for (int i = 0; i < d.nbf; i++) d.is_dir[fd[i]] = 1;
    }
}

// Pattern of the element connectivity over a subset of elements in a local numbering.
static void element_pattern(const Dofs& d, const std::vector<int64_t>& elems, int64_t n,
                            const std::vector<int64_t>& l_of_elemdof, Csr& pat) {
  // dof -> element incidence
  std::vector<int64_t> cnt(n + 1, 0);
  const int nb = d.nb;
  for (size_t i = 0; i < elems.size(); i++)
    for (int a = 0; a < nb; a++) cnt[l_of_elemdof[i * nb + a] + 1]++;
  for (int64_t r = 0; r < n; r++) cnt[r + 1] += cnt[r];
  std::vector<int64_t> inc(cnt[n]);
  std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
  for (size_t i = 0; i < elems.size(); i++)
    for (int a = 0; a < nb; a++) inc[fill[l_of_elemdof[i * nb + a]]++] = int64_t(i);
  pat.n = n;
  pat.ptr.assign(n + 1, 0);
  std::vector<int64_t> mark(n, -1);
  std::vector<int32_t> row;
  std::vector<int32_t> cols;
  cols.reserve(size_t(n) * (nb == 4 ? 16 : 40));
  for (int64_t r = 0; r < n; r++) {
    row.clear();
    for (int64_t k = cnt[r]; k < cnt[r + 1]; k++) {
      const int64_t i = inc[k];
      for (int b = 0; b < nb; b++) {
        const int64_t c = l_of_elemdof[i * nb + b];
        if (mark[c] != r) { mark[c] = r; row.push_back(int32_t(c)); }
      }
    }
    std::sort(row.begin(), row.end());
    cols.insert(cols.end(), row.begin(), row.end());
    pat.ptr[r + 1] = int64_t(cols.size());
  }
  pat.col.swap(cols);
}

static inline int64_t face_key(int64_t a, int64_t b, int64_t c, int64_t nv) {
  if (a > b) std::swap(a, b);
  if (b > c) std::swap(b, c);
  if (a > b) std::swap(a, b);
  return (a * nv + b) * nv + c;
}

// Owner element of each tagged boundary face.
static std::vector<int64_t> face_owners(const Mesh& m) {
  std::vector<std::pair<int64_t, int64_t>> tf(size_t(m.ne) * 4);
  for (int64_t e = 0; e < m.ne; e++)
    for (int k = 0; k < 4; k++)
      tf[4 * e + k] = {face_key(m.tets[4 * e + kTetFace[k][0]], m.tets[4 * e + kTetFace[k][1]],
                                m.tets[4 * e + kTetFace[k][2]], m.nv), e};
  std::sort(tf.begin(), tf.end());
  const int64_t nf = int64_t(m.tag.size());
  std::vector<int64_t> own(nf, -1);
  for (int64_t f = 0; f < nf; f++) {
    const int64_t k = face_key(m.faces[3 * f], m.faces[3 * f + 1], m.faces[3 * f + 2], m.nv);
    auto it = std::lower_bound(tf.begin(), tf.end(), std::make_pair(k, int64_t(-1)));
    if (it != tf.end() && it->first == k) own[f] = it->second;
  }
  return own;
}

// Fold the homogeneous Dirichlet condition: identity rows and columns.
static void fold_dirichlet(Parts& P, const uint8_t* is_dir_local) {
  for (int64_t r = 0; r < P.pat.n; r++)
    for (int64_t k = P.pat.ptr[r]; k < P.pat.ptr[r + 1]; k++) {
      const int64_t c = P.pat.col[k];
      if (is_dir_local[r] || is_dir_local[c]) {
        P.K[k] = (r == c) ? 1.0 : 0.0;
        P.M[k] = 0.0;
        P.B[k] = 0.0;
      }
    }
}

static void add_element(Parts& P, const int64_t* ld, int nb, const double* Ke, const double* Me, cplx w) {
  for (int a = 0; a < nb; a++)
    for (int b = 0; b < nb; b++) {
      const int64_t k = P.pat.find(ld[a], ld[b]);
      P.K[k] += Ke[a * nb + b];
      P.M[k] += w * Me[a * nb + b];
    }
}

static void add_face(Parts& P, const int64_t* ld, int nbf, int order, double area, cplx w) {
  const RefTables& R = ref();
  for (int a = 0; a < nbf; a++)
    for (int b = 0; b < nbf; b++) {
      const int64_t k = P.pat.find(ld[a], ld[b]);
      P.B[k] += w * (area * R.F[order - 1][a][b]);
    }
}

// Row a of the element stiffness and unit mass of element e.
static void element_row(const Mesh& m, int order, int64_t e, int a, double* Kr, double* Mr) {
  double g[4][3];
  const double vol = tet_grads(m.xyz.data(), m.tets.data() + 4 * e, g);
  double G[4][4];
  for (int p = 0; p < 4; p++)
    for (int q = 0; q < 4; q++) G[p][q] = g[p][0] * g[q][0] + g[p][1] * g[q][1] + g[p][2] * g[q][2];
  const int o = order - 1, nb = order == 1 ? 4 : 10;
  const RefTables& R = ref();
  for (int b = 0; b < nb; b++) {
    double s = 0;
    for (int p = 0; p < 4; p++)
      for (int q = 0; q < 4; q++) s += G[p][q] * R.S[o][a][b][p][q];
    Kr[b] = vol * s;
    Mr[b] = vol * R.M[o][a][b];
  }
}

// Global K, M', B' assembled row by row (rows in parallel, each row's element
// contributions added in increasing element order: deterministic).
void assemble_global(const Mesh& m, const Dofs& d, Parts& A) {
  std::vector<int64_t> all(m.ne);
  std::iota(all.begin(), all.end(), 0);
  element_pattern(d, all, d.n, d.elem, A.pat);
  const int64_t nnz = A.pat.nnz();
  A.K.assign(nnz, 0.0);
  A.M.assign(nnz, 0.0);
  A.B.assign(nnz, 0.0);
  const int nb = d.nb;
  const int64_t n = d.n;
  std::vector<int64_t> iptr(n + 1, 0);
  for (int64_t q = 0; q < m.ne * nb; q++) iptr[d.elem[q] + 1]++;
  for (int64_t r = 0; r < n; r++) iptr[r + 1] += iptr[r];
  std::vector<int64_t> inc(iptr[n]);
  {
    std::vector<int64_t> fill(iptr.begin(), iptr.end() - 1);
    for (int64_t q = 0; q < m.ne * nb; q++) inc[fill[d.elem[q]]++] = q;   // (element, local node) pairs
  }
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t r = 0; r < n; r++) {
    double Kr[10], Mr[10];
    for (int64_t t = iptr[r]; t < iptr[r + 1]; t++) {
      const int64_t e = inc[t] / nb;
      const int a = int(inc[t] % nb);
      element_row(m, d.order, e, a, Kr, Mr);
      const cplx w = 1.0 / (m.c[e] * m.c[e]);
      for (int b = 0; b < nb; b++) {
        const int64_t k = A.pat.find(r, d.elem[nb * e + b]);
        A.K[k] += Kr[b];
        A.M[k] += w * Mr[b];
      }
    }
  }
  const std::vector<int64_t> own = face_owners(m);
  int64_t fd[6];
  for (size_t f = 0; f < m.tag.size(); f++) {
    if (m.tag[f] != 1) continue;
    d.face_dofs(m.faces.data() + 3 * f, fd);
    add_face(A, fd, d.nbf, d.order, tri_area(m.xyz.data(), m.faces.data() + 3 * f), 1.0 / m.c[own[f]]);
  }
  fold_dirichlet(A, d.is_dir.data());
}

// ---------------------------------------------------------------------------
void rcb_partition(const Mesh& m, int nparts, std::vector<int32_t>& part) {
  const int64_t ne = m.ne;
  std::vector<double> cen(size_t(ne) * 3);
  for (int64_t e = 0; e < ne; e++)
    for (int i = 0; i < 3; i++) {
      const double* x = m.xyz.data();
      const int32_t* t = m.tets.data() + 4 * e;
      cen[3 * e + i] = (((x[3 * t[0] + i] + x[3 * t[1] + i]) + x[3 * t[2] + i]) + x[3 * t[3] + i]) * 0.25;
    }
  part.assign(ne, 0);
  std::vector<int64_t> ids(ne);
  std::iota(ids.begin(), ids.end(), 0);
  struct Job { int64_t lo, hi; int p0, p1; };
  std::vector<Job> stack{{0, ne, 0, nparts}};
  while (!stack.empty()) {
    Job j = stack.back();
    stack.pop_back();
    if (j.p1 - j.p0 == 1) {
      for (int64_t k = j.lo; k < j.hi; k++) part[ids[k]] = j.p0;
      continue;
    }
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t k = j.lo; k < j.hi; k++)
      for (int i = 0; i < 3; i++) {
        lo[i] = std::min(lo[i], cen[3 * ids[k] + i]);
        hi[i] = std::max(hi[i], cen[3 * ids[k] + i]);
      }
    int ax = 0;
    for (int i = 1; i < 3; i++)
      if (hi[i] - lo[i] > hi[ax] - lo[ax]) ax = i;
    std::stable_sort(ids.begin() + j.lo, ids.begin() + j.hi, [&](int64_t a, int64_t b) {
      const double ca = cen[3 * a + ax], cb = cen[3 * b + ax];
      return ca < cb || (ca == cb && a < b);
    });
    const int pm = (j.p0 + j.p1) / 2;
    const double frac = double(pm - j.p0) / double(j.p1 - j.p0);
    const int64_t cut = j.lo + int64_t(std::llround(double(j.hi - j.lo) * frac));
    stack.push_back({cut, j.hi, pm, j.p1});
    stack.push_back({j.lo, cut, j.p0, pm});
  }
}

// ---------------------------------------------------------------------------
// Vertex -> element incidence (CSR).
static void vertex_elements(const Mesh& m, std::vector<int64_t>& vptr, std::vector<int64_t>& vel) {
  const int64_t nv = m.nv, ne = m.ne;
  vptr.assign(nv + 1, 0);
  vel.resize(size_t(ne) * 4);
  for (int64_t e = 0; e < ne; e++)
    for (int k = 0; k < 4; k++) vptr[m.tets[4 * e + k] + 1]++;
  for (int64_t v = 0; v < nv; v++) vptr[v + 1] += vptr[v];
  std::vector<int64_t> fill(vptr.begin(), vptr.end() - 1);
  for (int64_t e = 0; e < ne; e++)
    for (int k = 0; k < 4; k++) vel[fill[m.tets[4 * e + k]]++] = e;
}

// Elements of part i grown by `overlap` layers, each layer adding every element that
// shares a vertex with the current set; layer[v] = the layer at which vertex v entered
// (0 for the part itself).  in_e / layer are scratch (all clear on entry; the caller
// clears the entries of elems / verts afterwards).
static void grow_part(const Mesh& m, const std::vector<int64_t>& vptr, const std::vector<int64_t>& vel,
                      const std::vector<int32_t>& part, int i, int overlap, std::vector<int32_t>& layer,
                      std::vector<uint8_t>& in_e, std::vector<int64_t>& elems, std::vector<int64_t>& verts) {
  std::vector<int64_t> frontier;
  for (int64_t e = 0; e < m.ne; e++)
    if (part[e] == i) { elems.push_back(e); in_e[e] = 1; }
  for (int64_t e : elems)
    for (int k = 0; k < 4; k++) {
      const int32_t v = m.tets[4 * e + k];
      if (layer[v] < 0) { layer[v] = 0; verts.push_back(v); frontier.push_back(v); }
    }
  for (int l = 1; l <= overlap; l++) {
    std::vector<int64_t> newe;
    for (int64_t v : frontier)
      for (int64_t k = vptr[v]; k < vptr[v + 1]; k++) {
        const int64_t e = vel[k];
        if (!in_e[e]) { in_e[e] = 1; newe.push_back(e); }
      }
    frontier.clear();
    for (int64_t e : newe) {
      elems.push_back(e);
      for (int k = 0; k < 4; k++) {
        const int32_t v = m.tets[4 * e + k];
        if (layer[v] < 0) { layer[v] = l; verts.push_back(v); frontier.push_back(v); }
      }
    }
  }
  std::sort(elems.begin(), elems.end());
}

// Partition-of-unity weight chi = 1 - l / overlap of each dof (edge dofs: mean of the
// two end vertices).
static void pu_weights(const Dofs& d, int64_t nv, const std::vector<int32_t>& layer, int overlap,
                       const std::vector<int64_t>& dofs, std::vector<double>& chi) {
  auto chiv = [&](int64_t v) { return overlap == 0 ? 1.0 : 1.0 - double(layer[v]) / double(overlap); };
  chi.resize(dofs.size());
  for (size_t k = 0; k < dofs.size(); k++) {
    const int64_t g = dofs[k];
    if (g < nv) chi[k] = chiv(g);
    else {
      const int64_t key = d.edge_key[g - nv];
      chi[k] = 0.5 * (chiv(key / nv) + chiv(key % nv));
    }
  }
}

void build_subdomains(const Mesh& m, const Dofs& d, const std::vector<int32_t>& part, int nsub,
                      int overlap, std::vector<Subdomain>& subs) {
  const int64_t nv = m.nv, ne = m.ne;
  std::vector<int64_t> vptr, vel;
  vertex_elements(m, vptr, vel);
  // global boundary faces: sorted keys with tags
  std::vector<std::pair<int64_t, int8_t>> bkeys(m.tag.size());
  for (size_t f = 0; f < m.tag.size(); f++)
    bkeys[f] = {face_key(m.faces[3 * f], m.faces[3 * f + 1], m.faces[3 * f + 2], nv), m.tag[f]};
  std::sort(bkeys.begin(), bkeys.end());

  subs.assign(nsub, Subdomain());
  std::vector<double> chi_sum(d.n, 0.0);
  std::vector<std::vector<double>> chis(nsub);

#pragma omp parallel
  {
    std::vector<int32_t> layer(nv, -1);
    std::vector<uint8_t> in_e(ne, 0);
    std::vector<int64_t> loc(d.n, -1);
#pragma omp for schedule(dynamic, 1)
    for (int i = 0; i < nsub; i++) {
      Subdomain& S = subs[i];
      std::vector<int64_t> elems, verts;
      grow_part(m, vptr, vel, part, i, overlap, layer, in_e, elems, verts);
      // dofs
      std::vector<int64_t> dofs;
      dofs.reserve(elems.size() * 2);
      for (int64_t e : elems)
        for (int a = 0; a < d.nb; a++) dofs.push_back(d.elem[d.nb * e + a]);
      std::sort(dofs.begin(), dofs.end());
      dofs.erase(std::unique(dofs.begin(), dofs.end()), dofs.end());
      const int64_t ni = int64_t(dofs.size());
      std::vector<double> chi;
      pu_weights(d, nv, layer, overlap, dofs, chi);
      for (int64_t k = 0; k < ni; k++) loc[dofs[k]] = k;
      // local operator on the element pattern of Gamma_i
      std::vector<int64_t> ld(elems.size() * d.nb);
      for (size_t q = 0; q < elems.size(); q++)
        for (int a = 0; a < d.nb; a++) ld[q * d.nb + a] = loc[d.elem[d.nb * elems[q] + a]];
      element_pattern(d, elems, ni, ld, S.A.pat);
      const int64_t nnz = S.A.pat.nnz();
      S.A.K.assign(nnz, 0.0);
      S.A.M.assign(nnz, 0.0);
      S.A.B.assign(nnz, 0.0);
      double Ke[100], Me[100];
      for (size_t q = 0; q < elems.size(); q++) {
        element(m, d.order, elems[q], Ke, Me);
        const cplx c = m.c[elems[q]];
        add_element(S.A, ld.data() + q * d.nb, d.nb, Ke, Me, 1.0 / (c * c));
      }
      // faces of Gamma_i seen once: global ABC faces keep the ABC, artificial
      // interfaces get the same impedance, Dirichlet faces nothing.
      std::vector<std::pair<int64_t, int64_t>> fk(elems.size() * 4);
      for (size_t q = 0; q < elems.size(); q++)
        for (int k = 0; k < 4; k++) {
          const int32_t* t = m.tets.data() + 4 * elems[q];
          fk[4 * q + k] = {face_key(t[kTetFace[k][0]], t[kTetFace[k][1]], t[kTetFace[k][2]], nv),
                           int64_t(4 * q + k)};
        }
      std::sort(fk.begin(), fk.end());
      int64_t fd[6], lfd[6];
      for (size_t a = 0; a < fk.size();) {
        size_t b = a + 1;
        while (b < fk.size() && fk[b].first == fk[a].first) b++;
        if (b - a == 1) {
          auto it = std::lower_bound(bkeys.begin(), bkeys.end(), std::make_pair(fk[a].first, int8_t(-128)));
          const bool on_bdry = it != bkeys.end() && it->first == fk[a].first;
          const bool absorbing = !on_bdry || it->second == 1;
          if (absorbing) {
            const int64_t q = fk[a].second / 4, k = fk[a].second % 4;
            const int32_t* t = m.tets.data() + 4 * elems[q];
            const int32_t f3[3] = {t[kTetFace[k][0]], t[kTetFace[k][1]], t[kTetFace[k][2]]};
            d.face_dofs(f3, fd);
            for (int z = 0; z < d.nbf; z++) lfd[z] = loc[fd[z]];
            add_face(S.A, lfd, d.nbf, d.order, tri_area(m.xyz.data(), f3), 1.0 / m.c[elems[q]]);
          }
        }
        a = b;
      }
      std::vector<uint8_t> ldir(ni);
      for (int64_t k = 0; k < ni; k++) ldir[k] = d.is_dir[dofs[k]];
      fold_dirichlet(S.A, ldir.data());
      // reset scratch
      for (int64_t e : elems) in_e[e] = 0;
      for (int64_t v : verts) layer[v] = -1;
      for (int64_t k = 0; k < ni; k++) loc[dofs[k]] = -1;
      S.elems.swap(elems);
      S.dofs.swap(dofs);
      chis[i].swap(chi);
    }
  }
  for (int i = 0; i < nsub; i++)
    for (size_t k = 0; k < subs[i].dofs.size(); k++) chi_sum[subs[i].dofs[k]] += chis[i][k];
  for (int i = 0; i < nsub; i++) {
    subs[i].D.resize(subs[i].dofs.size());
    for (size_t k = 0; k < subs[i].dofs.size(); k++) subs[i].D[k] = chis[i][k] / chi_sum[subs[i].dofs[k]];
  }
}

// ---------------------------------------------------------------------------
// Coarse level: exact interpolation of the coarse Lagrange basis at the fine
// nodes (the fine mesh refines the coarse one, so each fine element's nodes are
// interpolated from its parent coarse element alone) and the Galerkin pieces
// E_K, E_M, E_B = sum over fine elements (faces) of Z_e^T X_e Z_e.
// ---------------------------------------------------------------------------
// Barycentric coordinates of p in a tet whose gradients g and first vertex x0 are known.
static inline void bary_from(const double g[4][3], const double* x0, const double* p, double l[4]) {
  double s = 0;
  for (int k = 1; k < 4; k++) {
    l[k] = g[k][0] * (p[0] - x0[0]) + g[k][1] * (p[1] - x0[1]) + g[k][2] * (p[2] - x0[2]);
    s += l[k];
  }
  l[0] = 1.0 - s;
}

// Interpolation weights of the coarse basis of element E at fine node `node` (zeroed
// on fine Dirichlet nodes and for removed coarse Dirichlet dofs; rounding noise below
// 1e-12 dropped: the exact weights are dyadic rationals).  g: gradients of E.
static void coarse_zrow(const HostProblem& P, int64_t E, const double g[4][3], int64_t node, double* out) {
  const Mesh& cm = P.cmesh;
  const Dofs& d = P.dofs;
  const Dofs& cd = P.cdofs;
  const int nb = d.nb;
  double l[4], phi[10];
  bary_from(g, cm.xyz.data() + 3 * int64_t(cm.tets[4 * E]), d.coord.data() + 3 * node, l);
  eval_basis(d.order, l, phi);
  for (int b = 0; b < nb; b++) {
    double v = phi[b];
    if (std::fabs(v) < 1e-12 || d.is_dir[node] || P.cfree[cd.elem[nb * E + b]] < 0) v = 0.0;
    out[b] = v;
  }
}

void build_coarse(HostProblem& P, bool keep_pieces) {
  const Mesh& m = P.mesh;
  const Mesh& cm = P.cmesh;
  const Dofs& d = P.dofs;
  build_dofs(cm, d.order, P.cdofs);
  const Dofs& cd = P.cdofs;
  P.cfree.assign(cd.n, -1);
  int64_t nH = 0;
  for (int64_t k = 0; k < cd.n; k++)
    if (!cd.is_dir[k]) P.cfree[k] = nH++;
  P.nH = nH;
  const int nb = d.nb;
  const int64_t ncE = cm.ne;
  auto zrow = [&](int64_t E, const double g[4][3], int64_t node, double* out) { coarse_zrow(P, E, g, node, out); };
  // Z rows: for every fine node, the lowest fine element containing it
  std::vector<int64_t> first_elem(d.n, -1);
  for (int64_t e = m.ne - 1; e >= 0; e--)
    for (int a = 0; a < nb; a++) first_elem[d.elem[nb * e + a]] = e;
  std::vector<double> zval(size_t(d.n) * nb);
#pragma omp parallel for schedule(static)
  for (int64_t g = 0; g < d.n; g++) {
    const int64_t E = P.parent[first_elem[g]];
    double gr[4][3];
    tet_grads(cm.xyz.data(), cm.tets.data() + 4 * E, gr);
    zrow(E, gr, g, zval.data() + size_t(g) * nb);
  }
  P.Z.n = d.n;
  P.Z.ptr.assign(d.n + 1, 0);
  P.Z.col.clear();
  P.Zv.clear();
  for (int64_t g = 0; g < d.n; g++) {
    const int64_t E = P.parent[first_elem[g]];
    std::pair<int32_t, double> row[10];
    int cnt = 0;
    for (int b = 0; b < nb; b++) {
      const double v = zval[size_t(g) * nb + b];
      if (v != 0.0) row[cnt++] = {int32_t(P.cfree[cd.elem[nb * E + b]]), v};
    }
    std::sort(row, row + cnt);
    for (int q = 0; q < cnt; q++) { P.Z.col.push_back(row[q].first); P.Zv.push_back(row[q].second); }
    P.Z.ptr[g + 1] = int64_t(P.Z.col.size());
  }
  std::vector<double>().swap(zval);
  // Z^T
  P.Zt.n = nH;
  P.Zt.ptr.assign(nH + 1, 0);
  for (int64_t k = 0; k < P.Z.nnz(); k++) P.Zt.ptr[P.Z.col[k] + 1]++;
  for (int64_t r = 0; r < nH; r++) P.Zt.ptr[r + 1] += P.Zt.ptr[r];
  P.Zt.col.resize(P.Z.nnz());
  P.Ztv.resize(P.Z.nnz());
  {
    std::vector<int64_t> fill(P.Zt.ptr.begin(), P.Zt.ptr.end() - 1);
    for (int64_t g = 0; g < d.n; g++)
      for (int64_t k = P.Z.ptr[g]; k < P.Z.ptr[g + 1]; k++) {
        const int64_t q = fill[P.Z.col[k]]++;
        P.Zt.col[q] = int32_t(g);
        P.Ztv[q] = P.Zv[k];
      }
  }
  // coarse pattern over free coarse dofs
  {
    std::vector<int64_t> all(cm.ne);
    std::iota(all.begin(), all.end(), 0);
    Csr full;
    element_pattern(cd, all, cd.n, cd.elem, full);
    P.E.pat.n = nH;
    P.E.pat.ptr.assign(nH + 1, 0);
    P.E.pat.col.clear();
    for (int64_t r = 0; r < cd.n; r++) {
      if (P.cfree[r] < 0) continue;
      for (int64_t k = full.ptr[r]; k < full.ptr[r + 1]; k++)
        if (P.cfree[full.col[k]] >= 0) P.E.pat.col.push_back(int32_t(P.cfree[full.col[k]]));
      P.E.pat.ptr[P.cfree[r] + 1] = int64_t(P.E.pat.col.size());
    }
  }
  // fine elements and absorbing faces grouped by coarse parent
  std::vector<int64_t> cptr(ncE + 1, 0), kids(m.ne);
  for (int64_t e = 0; e < m.ne; e++) cptr[P.parent[e] + 1]++;
  for (int64_t E = 0; E < ncE; E++) cptr[E + 1] += cptr[E];
  {
    std::vector<int64_t> fill(cptr.begin(), cptr.end() - 1);
    for (int64_t e = 0; e < m.ne; e++) kids[fill[P.parent[e]]++] = e;
  }
  const std::vector<int64_t> own = face_owners(m);
  std::vector<int64_t> fptr(ncE + 1, 0), fids;
  for (size_t f = 0; f < m.tag.size(); f++)
    if (m.tag[f] == 1) fptr[P.parent[own[f]] + 1]++;
  for (int64_t E = 0; E < ncE; E++) fptr[E + 1] += fptr[E];
  fids.resize(fptr[ncE]);
  {
    std::vector<int64_t> fill(fptr.begin(), fptr.end() - 1);
    for (size_t f = 0; f < m.tag.size(); f++)
      if (m.tag[f] == 1) fids[fill[P.parent[own[f]]]++] = int64_t(f);
  }
  // Galerkin pieces per coarse element: sum over its fine children of Z_e^T X_e Z_e
  const size_t nb2 = size_t(nb) * nb;
  std::vector<double> EK(size_t(ncE) * nb2);
  std::vector<cplx> EM(size_t(ncE) * nb2), EB(size_t(ncE) * nb2);
  const RefTables& R = ref();
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t E = 0; E < ncE; E++) {
    double gr[4][3];
    tet_grads(cm.xyz.data(), cm.tets.data() + 4 * E, gr);
    double* ek = EK.data() + size_t(E) * nb2;
    cplx* em = EM.data() + size_t(E) * nb2;
    cplx* eb = EB.data() + size_t(E) * nb2;
    for (size_t q = 0; q < nb2; q++) { ek[q] = 0; em[q] = 0; eb[q] = 0; }
    double Ke[100], Me[100], Z[100], T1[100], T2[100];
    for (int64_t q = cptr[E]; q < cptr[E + 1]; q++) {
      const int64_t e = kids[q];
      element(m, d.order, e, Ke, Me);
      for (int a = 0; a < nb; a++) zrow(E, gr, d.elem[nb * e + a], Z + a * nb);
      for (int a = 0; a < nb; a++)
        for (int b = 0; b < nb; b++) {
          double sk = 0, sm = 0;
          for (int c = 0; c < nb; c++) { sk += Ke[a * nb + c] * Z[c * nb + b]; sm += Me[a * nb + c] * Z[c * nb + b]; }
          T1[a * nb + b] = sk;
          T2[a * nb + b] = sm;
        }
      const cplx w = 1.0 / (m.c[e] * m.c[e]);
      for (int a = 0; a < nb; a++)
        for (int b = 0; b < nb; b++) {
          double sk = 0, sm = 0;
          for (int c = 0; c < nb; c++) { sk += Z[c * nb + a] * T1[c * nb + b]; sm += Z[c * nb + a] * T2[c * nb + b]; }
          ek[a * nb + b] += sk;
          em[a * nb + b] += w * sm;
        }
    }
    for (int64_t q = fptr[E]; q < fptr[E + 1]; q++) {
      const int64_t f = fids[q];
      const int64_t e = own[f];
      int64_t fd[6];
      d.face_dofs(m.faces.data() + 3 * f, fd);
      double Zf[60];
      for (int z = 0; z < d.nbf; z++) zrow(E, gr, fd[z], Zf + z * nb);
      const double area = tri_area(m.xyz.data(), m.faces.data() + 3 * f);
      const cplx w = 1.0 / m.c[e];
      for (int a = 0; a < nb; a++)
        for (int b = 0; b < nb; b++) {
          double sacc = 0;
          for (int p = 0; p < d.nbf; p++)
            for (int r = 0; r < d.nbf; r++)
              sacc += Zf[p * nb + a] * area * R.F[d.order - 1][p][r] * Zf[r * nb + b];
          eb[a * nb + b] += w * sacc;
        }
    }
  }
  const int64_t nnzE = P.E.pat.nnz();
  P.E.K.assign(nnzE, 0.0);
  P.E.M.assign(nnzE, 0.0);
  P.E.B.assign(nnzE, 0.0);
  for (int64_t E = 0; E < ncE; E++) {
    int64_t cfd[10];
    for (int b = 0; b < nb; b++) cfd[b] = P.cfree[cd.elem[nb * E + b]];
    for (int a = 0; a < nb; a++) {
      if (cfd[a] < 0) continue;
      for (int b = 0; b < nb; b++) {
        if (cfd[b] < 0) continue;
        const int64_t k = P.E.pat.find(cfd[a], cfd[b]);
        const size_t q = size_t(E) * nb2 + a * nb + b;
        P.E.K[k] += EK[q];
        P.E.M[k] += EM[q];
        P.E.B[k] += EB[q];
      }
    }
  }
  if (keep_pieces) {
    P.cEK.swap(EK);
    P.cEM.swap(EM);
    P.cEB.swap(EB);
  }
}

// Coarse level of the iterative coarse solve: one-level ORAS on the coarse mesh with
// the fine partition carried over (a coarse element joins the part holding most of its
// fine children; ties: lowest part), the fine overlap and partition-of-unity recipe
// applied to the coarse mesh, and local operators E_i = sum of the Galerkin pieces of
// the coarse elements of Gamma_H,i plus, on its artificial interfaces, the Galerkin
// projection of the fine absorbing term (fine faces on the coarse face, coefficient of
// the fine element inside).  Coarse Dirichlet dofs are identity rows with weight 0.
void build_coarse_subdomains(HostProblem& P, const std::vector<int32_t>& part, int nsub, int overlap) {
  const Mesh& m = P.mesh;
  const Mesh& cm = P.cmesh;
  const Dofs& d = P.dofs;
  const Dofs& cd = P.cdofs;
  const int nb = d.nb;
  const size_t nb2 = size_t(nb) * nb;
  const int64_t ncE = cm.ne, nvH = cm.nv;
  std::vector<int64_t> cptr(ncE + 1, 0), kids(m.ne);
  for (int64_t e = 0; e < m.ne; e++) cptr[P.parent[e] + 1]++;
  for (int64_t E = 0; E < ncE; E++) cptr[E + 1] += cptr[E];
  {
    std::vector<int64_t> fill(cptr.begin(), cptr.end() - 1);
    for (int64_t e = 0; e < m.ne; e++) kids[fill[P.parent[e]]++] = e;
  }
  P.cpart.assign(ncE, 0);
  for (int64_t E = 0; E < ncE; E++) {
    int32_t best = -1, bestc = 0;
    for (int64_t q = cptr[E]; q < cptr[E + 1]; q++) {
      const int32_t pq = part[kids[q]];
      int32_t c = 0;
      for (int64_t r = cptr[E]; r < cptr[E + 1]; r++) c += part[kids[r]] == pq;
      if (c > bestc || (c == bestc && pq < best)) { best = pq; bestc = c; }
    }
    P.cpart[E] = best < 0 ? 0 : best;
  }
  std::vector<int64_t> vptr, vel;
  vertex_elements(cm, vptr, vel);
  std::vector<std::pair<int64_t, int8_t>> bkeys(cm.tag.size());
  for (size_t f = 0; f < cm.tag.size(); f++)
    bkeys[f] = {face_key(cm.faces[3 * f], cm.faces[3 * f + 1], cm.faces[3 * f + 2], nvH), cm.tag[f]};
  std::sort(bkeys.begin(), bkeys.end());
  const RefTables& R = ref();
  P.csubs.assign(nsub, Subdomain());
  std::vector<std::vector<double>> chis(nsub);
#pragma omp parallel
  {
    std::vector<int32_t> layer(nvH, -1);
    std::vector<uint8_t> in_e(ncE, 0);
    std::vector<int64_t> loc(cd.n, -1);
#pragma omp for schedule(dynamic, 1)
    for (int i = 0; i < nsub; i++) {
      Subdomain& S = P.csubs[i];
      std::vector<int64_t> elems, verts;
      grow_part(cm, vptr, vel, P.cpart, i, overlap, layer, in_e, elems, verts);
      std::vector<int64_t> dofs;
      for (int64_t E : elems)
        for (int a = 0; a < nb; a++) dofs.push_back(cd.elem[nb * E + a]);
      std::sort(dofs.begin(), dofs.end());
      dofs.erase(std::unique(dofs.begin(), dofs.end()), dofs.end());
      const int64_t ni = int64_t(dofs.size());
      std::vector<double> chi;
      pu_weights(cd, nvH, layer, overlap, dofs, chi);
      for (int64_t k = 0; k < ni; k++) loc[dofs[k]] = k;
      std::vector<int64_t> ld(elems.size() * nb);
      for (size_t q = 0; q < elems.size(); q++)
        for (int a = 0; a < nb; a++) ld[q * nb + a] = loc[cd.elem[nb * elems[q] + a]];
      element_pattern(cd, elems, ni, ld, S.A.pat);
      const int64_t nnz = S.A.pat.nnz();
      S.A.K.assign(nnz, 0.0);
      S.A.M.assign(nnz, 0.0);
      S.A.B.assign(nnz, 0.0);
      for (size_t q = 0; q < elems.size(); q++) {
        const size_t o = size_t(elems[q]) * nb2;
        for (int a = 0; a < nb; a++)
          for (int b = 0; b < nb; b++) {
            const int64_t k = S.A.pat.find(ld[q * nb + a], ld[q * nb + b]);
            S.A.K[k] += P.cEK[o + a * nb + b];
            S.A.M[k] += P.cEM[o + a * nb + b];
            S.A.B[k] += P.cEB[o + a * nb + b];
          }
      }
      // coarse faces of Gamma_H,i seen once and not on the global boundary
      std::vector<std::pair<int64_t, int64_t>> fk(elems.size() * 4);
      for (size_t q = 0; q < elems.size(); q++)
        for (int k = 0; k < 4; k++) {
          const int32_t* t = cm.tets.data() + 4 * elems[q];
          fk[4 * q + k] = {face_key(t[kTetFace[k][0]], t[kTetFace[k][1]], t[kTetFace[k][2]], nvH), int64_t(4 * q + k)};
        }
      std::sort(fk.begin(), fk.end());
      for (size_t a = 0; a < fk.size();) {
        size_t b = a + 1;
        while (b < fk.size() && fk[b].first == fk[a].first) b++;
        if (b - a == 1) {
          auto it = std::lower_bound(bkeys.begin(), bkeys.end(), std::make_pair(fk[a].first, int8_t(-128)));
          const bool on_bdry = it != bkeys.end() && it->first == fk[a].first;
          if (!on_bdry) {
            const size_t q = size_t(fk[a].second / 4);
            const int kf = int(fk[a].second % 4);
            const int64_t E = elems[q];
            double gr[4][3];
            tet_grads(cm.xyz.data(), cm.tets.data() + 4 * E, gr);
            const double* x0 = cm.xyz.data() + 3 * int64_t(cm.tets[4 * E]);
            cplx piece[100];
            for (size_t z = 0; z < nb2; z++) piece[z] = 0.0;
            for (int64_t c = cptr[E]; c < cptr[E + 1]; c++) {
              const int64_t e = kids[c];
              const int32_t* t = m.tets.data() + 4 * e;
              for (int fq = 0; fq < 4; fq++) {
                const int32_t f3[3] = {t[kTetFace[fq][0]], t[kTetFace[fq][1]], t[kTetFace[fq][2]]};
                bool on = true;
                for (int v = 0; v < 3 && on; v++) {
                  double l[4];
                  bary_from(gr, x0, m.xyz.data() + 3 * int64_t(f3[v]), l);
                  on = std::fabs(l[kf]) < 1e-9;
                }
                if (!on) continue;
                int64_t fd[6];
                d.face_dofs(f3, fd);
                double Zf[60];
                for (int z = 0; z < d.nbf; z++) coarse_zrow(P, E, gr, fd[z], Zf + z * nb);
                const double area = tri_area(m.xyz.data(), f3);
                const cplx w = 1.0 / m.c[e];
                for (int aa = 0; aa < nb; aa++)
                  for (int bb = 0; bb < nb; bb++) {
                    double sacc = 0;
                    for (int pp = 0; pp < d.nbf; pp++)
                      for (int rr = 0; rr < d.nbf; rr++)
                        sacc += Zf[pp * nb + aa] * area * R.F[d.order - 1][pp][rr] * Zf[rr * nb + bb];
                    piece[aa * nb + bb] += w * sacc;
                  }
              }
            }
            for (int aa = 0; aa < nb; aa++)
              for (int bb = 0; bb < nb; bb++) {
                const int64_t k = S.A.pat.find(ld[q * nb + aa], ld[q * nb + bb]);
                S.A.B[k] += piece[aa * nb + bb];
              }
          }
        }
        a = b;
      }
      std::vector<uint8_t> ldir(ni);
      for (int64_t k = 0; k < ni; k++) ldir[k] = cd.is_dir[dofs[k]];
      fold_dirichlet(S.A, ldir.data());
      for (int64_t E : elems) in_e[E] = 0;
      for (int64_t v : verts) layer[v] = -1;
      for (int64_t k = 0; k < ni; k++) loc[dofs[k]] = -1;
      S.elems.swap(elems);
      S.dofs.swap(dofs);
      chis[i].swap(chi);
    }
  }
  std::vector<double> chi_sum(cd.n, 0.0);
  for (int i = 0; i < nsub; i++)
    for (size_t k = 0; k < P.csubs[i].dofs.size(); k++) chi_sum[P.csubs[i].dofs[k]] += chis[i][k];
  P.cgidx.assign(nsub, {});
  for (int i = 0; i < nsub; i++) {
    Subdomain& S = P.csubs[i];
    S.D.resize(S.dofs.size());
    P.cgidx[i].resize(S.dofs.size());
    for (size_t k = 0; k < S.dofs.size(); k++) {
      const int64_t g = S.dofs[k];
      const bool free = P.cfree[g] >= 0;
      S.D[k] = free ? chis[i][k] / chi_sum[g] : 0.0;
      P.cgidx[i][k] = free ? P.cfree[g] : 0;
    }
  }
  std::vector<double>().swap(P.cEK);
  std::vector<cplx>().swap(P.cEM);
  std::vector<cplx>().swap(P.cEB);
}

bool locate_point(const Mesh& m, const double* p, int64_t& elem, double lam[4]) {
  for (int64_t e = 0; e < m.ne; e++) {
    const int32_t* t = m.tets.data() + 4 * e;
    bool out = false;
    for (int i = 0; i < 3 && !out; i++) {
      double lo = 1e300, hi = -1e300;
      for (int k = 0; k < 4; k++) {
        lo = std::min(lo, m.xyz[3 * int64_t(t[k]) + i]);
        hi = std::max(hi, m.xyz[3 * int64_t(t[k]) + i]);
      }
      out = p[i] < lo - 1e-12 || p[i] > hi + 1e-12;
    }
    if (out) continue;
    barycentric(m.xyz.data(), t, p, lam);
    if (lam[0] >= -1e-12 && lam[1] >= -1e-12 && lam[2] >= -1e-12 && lam[3] >= -1e-12) {
      elem = e;
      return true;
    }
  }
  return false;
}

}  // namespace hz
