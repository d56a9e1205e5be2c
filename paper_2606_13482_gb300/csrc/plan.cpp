// Host-side planning: geometry, octree, spline algebra, moments, lists.
// See plan.hpp for the paper passages each part follows.
#include "plan.hpp"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <unordered_map>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace efie {

static const int S_REMOVE[7] = {0, 0, 0, 1, 1, 2, 2};  // Table I, index p

[[noreturn]] static void fail(int code, const std::string& m) { throw EfieError{code, m}; }

// ------------------------------------------------------------------ geometry
// Sec. II: RWG without edge-length normalization; c+ is the triangle whose CCW
// cycle runs lo -> hi along the edge (lo < hi).
static void build_geometry(Geometry& g, const double* xyz, int64_t nv, const int32_t* tri,
                           int64_t nt) {
  if (nv < 4 || nt < 4) fail(-1, "mesh too small");
  g.nv = nv;
  g.nt = nt;
  g.V.assign(xyz, xyz + 3 * nv);
  g.T.assign(tri, tri + 3 * nt);
  g.area.resize(nt);
  g.cen.resize(3 * nt);
  for (int64_t t = 0; t < nt; ++t) {
    for (int k = 0; k < 3; ++k)
      if (g.T[3 * t + k] < 0 || g.T[3 * t + k] >= nv) fail(-1, "triangle vertex id out of range");
    const double* a = &g.V[3 * g.T[3 * t]];
    const double* b = &g.V[3 * g.T[3 * t + 1]];
    const double* c = &g.V[3 * g.T[3 * t + 2]];
    double e1[3], e2[3], n[3];
    for (int d = 0; d < 3; ++d) {
      e1[d] = b[d] - a[d];
      e2[d] = c[d] - a[d];
    }
    n[0] = e1[1] * e2[2] - e1[2] * e2[1];
    n[1] = e1[2] * e2[0] - e1[0] * e2[2];
    n[2] = e1[0] * e2[1] - e1[1] * e2[0];
    double nn = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    if (!(nn > 1e-300)) fail(-1, "degenerate triangle " + std::to_string(t));
    g.area[t] = 0.5 * nn;
    for (int d = 0; d < 3; ++d) g.cen[3 * t + d] = (a[d] + b[d] + c[d]) / 3.0;
  }
  struct HalfEdge {
    int64_t key;
    int32_t t;
    int32_t fwd;
    int32_t w;
  };
  std::vector<HalfEdge> he(3 * nt);
  for (int64_t t = 0; t < nt; ++t)
    for (int k = 0; k < 3; ++k) {
      int32_t u = g.T[3 * t + k], v = g.T[3 * t + (k + 1) % 3], w = g.T[3 * t + (k + 2) % 3];
      int64_t lo = std::min(u, v), hi = std::max(u, v);
      if (lo == hi) fail(-1, "repeated vertex in a triangle");
      he[3 * t + k] = {lo * nv + hi, (int32_t)t, u < v ? 1 : 0, w};
    }
  std::sort(he.begin(), he.end(), [](const HalfEdge& a, const HalfEdge& b) {
    return a.key != b.key ? a.key < b.key : a.t < b.t;
  });
  g.N = 0;
  for (size_t i = 0; i < he.size();) {
    size_t j = i;
    while (j < he.size() && he[j].key == he[i].key) ++j;
    if (j - i != 2) fail(-1, "mesh is not a closed 2-manifold (edge shared by " +
                                 std::to_string(j - i) + " triangles)");
    if (he[i].fwd == he[i + 1].fwd) fail(-1, "inconsistent triangle orientation");
    const HalfEdge& pl = he[i].fwd ? he[i] : he[i + 1];
    const HalfEdge& mi = he[i].fwd ? he[i + 1] : he[i];
    g.edge.push_back((int32_t)(he[i].key / nv));
    g.edge.push_back((int32_t)(he[i].key % nv));
    g.tri_pm.push_back(pl.t);
    g.tri_pm.push_back(mi.t);
    g.free_pm.push_back(pl.w);
    g.free_pm.push_back(mi.w);
    ++g.N;
    i = j;
  }
}

// ------------------------------------------------------------------ splines
std::vector<double> open_knots(double lo, double hi, int ns, int p) {
  int m = ns - p;
  std::vector<double> U;
  for (int i = 0; i <= p; ++i) U.push_back(lo);
  for (int i = 1; i < m; ++i) U.push_back(lo + (hi - lo) * i / m);
  for (int i = 0; i <= p; ++i) U.push_back(hi);
  return U;
}

// All B-splines of U at x (Cox-de Boor), spans half-open except the last
// non-empty one (closed), so x = right end is covered.
static void basis_all(const std::vector<double>& U, int p, double x, std::vector<double>& out) {
  int nk = (int)U.size();
  int last = -1;
  for (int i = 0; i + 1 < nk; ++i)
    if (U[i] < U[i + 1]) last = i;
  std::vector<double> N(nk - 1, 0.0);
  for (int i = 0; i + 1 < nk; ++i)
    if (U[i] < U[i + 1]) {
      bool in = (x >= U[i]) && (i == last ? x <= U[i + 1] : x < U[i + 1]);
      N[i] = in ? 1.0 : 0.0;
    }
  for (int q = 1; q <= p; ++q) {
    for (int i = 0; i + q + 1 < nk; ++i) {
      double t = 0.0;
      double d1 = U[i + q] - U[i];
      if (d1 > 0) t += (x - U[i]) / d1 * N[i];
      double d2 = U[i + q + 1] - U[i + 1];
      if (d2 > 0) t += (U[i + q + 1] - x) / d2 * N[i + 1];
      N[i] = t;
    }
  }
  out.assign(N.begin(), N.begin() + (nk - p - 1));
}

// Boehm insertion (Sec. IV-B): with u_k <= ub < u_{k+1}, new coefficients
// w_i' = a_i w_i + (1 - a_i) w_{i-1}, a_i = (ub - u_i)/(u_{i+p} - u_i) on
// k-p+1..k, 1 below, 0 above.
static void insert_knot(std::vector<double>& U, int p, std::vector<double>& w, double ub) {
  int k = (int)(std::upper_bound(U.begin(), U.end(), ub) - U.begin()) - 1;
  int n = (int)w.size();
  std::vector<double> wb(n + 1);
  for (int i = 0; i <= n; ++i) {
    if (i <= k - p)
      wb[i] = w[i];
    else if (i >= k + 1)
      wb[i] = w[i - 1];
    else {
      double a = (ub - U[i]) / (U[i + p] - U[i]);
      wb[i] = a * w[i] + (1.0 - a) * w[i - 1];
    }
  }
  U.insert(U.begin() + k + 1, ub);
  w.swap(wb);
}

static void refine_to(std::vector<double>& U, int p, std::vector<double>& w,
                      const std::vector<double>& target) {
  std::vector<double> t = target;
  std::sort(t.begin(), t.end());
  for (size_t i = 0; i < t.size();) {
    size_t j = i;
    while (j < t.size() && t[j] == t[i]) ++j;
    long need = (long)(j - i) - (long)std::count(U.begin(), U.end(), t[i]);
    for (long r = 0; r < need; ++r) insert_knot(U, p, w, t[i]);
    i = j;
  }
}

std::vector<double> restriction_matrix(const std::vector<double>& Up,
                                       const std::vector<double>& Uc, int p, int* rows,
                                       int* cols) {
  double a = Uc.front(), b = Uc.back();
  int nsp = (int)Up.size() - p - 1, nsc = (int)Uc.size() - p - 1;
  std::vector<double> target;
  for (double t : Up)
    if (t < a || t > b) target.push_back(t);
  for (double t : Uc) target.push_back(t);
  std::vector<double> C((size_t)nsp * nsc);
  for (int j = 0; j < nsp; ++j) {
    std::vector<double> U = Up, w(nsp, 0.0);
    w[j] = 1.0;
    refine_to(U, p, w, target);
    int k0 = (int)(std::lower_bound(U.begin(), U.end(), a) - U.begin());
    for (int i = 0; i < nsc + p + 1; ++i)
      if (U[k0 + i] != Uc[i]) fail(-1, "child knots not nested in the parent knot vector");
    for (int i = 0; i < nsc; ++i) C[(size_t)j * nsc + i] = w[k0 + i];
  }
  *rows = nsp;
  *cols = nsc;
  return C;
}

// Dense LU with partial pivoting: solves A X = B in place (A n x n, B n x m).
static void lu_solve(std::vector<double> A, int n, std::vector<double>& B, int m) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[(size_t)r * n + c]) > std::fabs(A[(size_t)piv * n + c])) piv = r;
    if (A[(size_t)piv * n + c] == 0.0) fail(-1, "singular sampling matrix");
    if (piv != c) {
      for (int k = 0; k < n; ++k) std::swap(A[(size_t)c * n + k], A[(size_t)piv * n + k]);
      for (int k = 0; k < m; ++k) std::swap(B[(size_t)c * m + k], B[(size_t)piv * m + k]);
    }
    for (int r = c + 1; r < n; ++r) {
      double f = A[(size_t)r * n + c] / A[(size_t)c * n + c];
      if (f == 0.0) continue;
      for (int k = c; k < n; ++k) A[(size_t)r * n + k] -= f * A[(size_t)c * n + k];
      for (int k = 0; k < m; ++k) B[(size_t)r * m + k] -= f * B[(size_t)c * m + k];
    }
  }
  for (int c = n - 1; c >= 0; --c) {
    for (int k = 0; k < m; ++k) {
      double s = B[(size_t)c * m + k];
      for (int j = c + 1; j < n; ++j) s -= A[(size_t)c * n + j] * B[(size_t)j * m + k];
      B[(size_t)c * m + k] = s / A[(size_t)c * n + c];
    }
  }
}

// P = B_stab^{-1} S (Sec. V-B): stabilized knots drop the first and last
// s_remove interior knots; S by knot insertion; B_stab[m][k] = b_m(x_k) at s_hat
// equispaced points including both domain ends.
static void projector(int sp, int p, std::vector<double>& P, int* shat_out) {
  std::vector<double> Ue = open_knots(0.0, (double)(sp - p), sp, p);
  int r = S_REMOVE[p];
  std::vector<double> Us;
  for (int i = 0; i <= p; ++i) Us.push_back(Ue.front());
  for (size_t i = p + 1 + r; i + p + 1 + r < Ue.size(); ++i) Us.push_back(Ue[i]);
  for (int i = 0; i <= p; ++i) Us.push_back(Ue.back());
  int ns = (int)Us.size() - p - 1;
  // S[j][i]: equidistant coefficients of stabilized spline j
  std::vector<double> S((size_t)ns * sp);
  for (int j = 0; j < ns; ++j) {
    std::vector<double> U = Us, w(ns, 0.0);
    w[j] = 1.0;
    refine_to(U, p, w, Ue);
    for (int i = 0; i < sp; ++i) S[(size_t)j * sp + i] = w[i];
  }
  std::vector<double> B((size_t)ns * ns), row;
  for (int kk = 0; kk < ns; ++kk) {
    double x = Ue.front() + (Ue.back() - Ue.front()) * kk / (ns - 1);
    basis_all(Us, p, x, row);
    for (int m = 0; m < ns; ++m) B[(size_t)m * ns + kk] = row[m];
  }
  lu_solve(B, ns, S, sp);
  P = S;
  *shat_out = ns;
}

void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
  // Newton iteration on the Legendre polynomial P_n (three-term recurrence)
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double pn = (n == 1) ? z : p1;
      double pm = (n == 1) ? 1.0 : p0;
      dp = n * (z * pn - pm) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double pn = (n == 1) ? z : p1;
      double pm = (n == 1) ? 1.0 : p0;
      dp = n * (z * pn - pm) / (z * z - 1.0);
    }
    x[n - 1 - i] = 0.5 * (z + 1.0);
    w[n - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);  // (2/((1-z^2)P'^2)) / 2
  }
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::sort(idx.begin(), idx.end(), [&](int a, int b) { return x[a] < x[b]; });
  std::vector<double> xs(n), ws(n);
  for (int i = 0; i < n; ++i) {
    xs[i] = x[idx[i]];
    ws[i] = w[idx[i]];
  }
  x.swap(xs);
  w.swap(ws);
}

// ------------------------------------------------------------------ octree
static uint64_t spread3(uint64_t v) {
  v &= 0x1fffff;
  v = (v | v << 32) & 0x1f00000000ffffULL;
  v = (v | v << 16) & 0x1f0000ff0000ffULL;
  v = (v | v << 8) & 0x100f00f00f00f00fULL;
  v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
  v = (v | v << 2) & 0x1249249249249249ULL;
  return v;
}
static uint64_t morton(int64_t i, int64_t j, int64_t k) {
  return spread3((uint64_t)i) | (spread3((uint64_t)j) << 1) | (spread3((uint64_t)k) << 2);
}
static int64_t find_code(const std::vector<uint64_t>& codes, uint64_t c) {
  auto it = std::lower_bound(codes.begin(), codes.end(), c);
  if (it == codes.end() || *it != c) return -1;
  return it - codes.begin();
}

static void box_of(const Plan& P, const double* x, int level, int64_t* ijk) {
  double h = P.root_edge / (double)(1LL << level);
  int64_t nb = 1LL << level;
  for (int d = 0; d < 3; ++d) {
    int64_t i = (int64_t)std::floor((x[d] - P.root_lo[d]) / h);
    ijk[d] = std::min<int64_t>(std::max<int64_t>(i, 0), nb - 1);
  }
}

// ------------------------------------------------------------------ moments
namespace {
struct Poly {
  int n = 0;
  double v[24][3];
};

void split(const Poly& P, int axis, double val, Poly& L, Poly& R) {
  L.n = R.n = 0;
  for (int i = 0; i < P.n; ++i) {
    const double* a = P.v[i];
    const double* b = P.v[(i + 1) % P.n];
    double sa = a[axis] - val, sb = b[axis] - val;
    if (sa <= 0) { std::memcpy(L.v[L.n++], a, sizeof(double) * 3); }
    if (sa >= 0) { std::memcpy(R.v[R.n++], a, sizeof(double) * 3); }
    if ((sa < 0 && sb > 0) || (sb < 0 && sa > 0)) {
      double t = sa / (sa - sb);
      double x[3];
      for (int d = 0; d < 3; ++d) x[d] = a[d] + t * (b[d] - a[d]);
      x[axis] = val;
      std::memcpy(L.v[L.n++], x, sizeof(x));
      std::memcpy(R.v[R.n++], x, sizeof(x));
    }
  }
}

struct LeafKnots {
  int p, sp;
  double lo[3], delta;
  std::vector<double> U[3];
};

int find_span(const std::vector<double>& U, int p, int ns, double x) {
  if (x >= U[ns]) return ns - 1;
  if (x <= U[p]) return p;
  int lo = p, hi = ns;
  while (hi - lo > 1) {
    int mid = (lo + hi) / 2;
    if (x < U[mid]) hi = mid; else lo = mid;
  }
  return lo;
}

// The nonzero B-splines N_{i-p..i}(x) in span i come from the triangular
// recursion (Cox-de Boor).  Its denominators
// (x - U[i+1-j+r]) + (U[i+r+1] - x) = U[i+r+1] - U[i+1-j+r] do not depend on
// x and are positive for a nonempty span, so their reciprocals are taken once
// per span.
static void span_recip(const std::vector<double>& U, int p, int i, double* inv) {
  int k = 0;
  for (int j = 1; j <= p; ++j)
    for (int r = 0; r < j; ++r) inv[k++] = 1.0 / (U[i + r + 1] - U[i + 1 - j + r]);
}

// N[0..p] = N_{i-p..i}(x), with the reciprocals of span_recip
static inline void basis_nz_r(const std::vector<double>& U, int p, int i, const double* inv, double x,
                              double* N) {
  double left[8], right[8];
  N[0] = 1.0;
  int k = 0;
  for (int j = 1; j <= p; ++j) {
    left[j] = x - U[i + 1 - j];
    right[j] = U[i + j] - x;
    double saved = 0.0;
    for (int r = 0; r < j; ++r) {
      double tmp = N[r] * inv[k++];
      N[r] = saved + right[r + 1] * tmp;
      saved = left[j - r] * tmp;
    }
    N[j] = saved;
  }
}

// T[i0][i1][c][i2] = sum_q NN[i0 p1 + i1][q] F[q][c][i2]: the sum over a
// piece's quadrature points of the rank-one products N_i0 N_i1 (f_c N_i2),
// one output row at a time so that the row stays in registers.
template <int P1>
static void contract_rows(const double* __restrict NN, const double* __restrict F, int Q, int ld,
                          double* __restrict T) {
  constexpr int W = 4 * P1;
  for (int ii = 0; ii < P1 * P1; ++ii) {
    double row[W];
    for (int j = 0; j < W; ++j) row[j] = 0.0;
    const double* nn = NN + (size_t)ii * ld;
    for (int q = 0; q < Q; ++q) {
      const double a = nn[q];
      const double* f = F + (size_t)q * W;
      for (int j = 0; j < W; ++j) row[j] += a * f[j];
    }
    for (int j = 0; j < W; ++j) T[ii * W + j] = row[j];
  }
}
using contract_fn = void (*)(const double*, const double*, int, int, double*);
static contract_fn contract_for(int p1) {
  switch (p1) {
    case 2: return contract_rows<2>;
    case 3: return contract_rows<3>;
    case 4: return contract_rows<4>;
    case 5: return contract_rows<5>;
    case 6: return contract_rows<6>;
    default: return contract_rows<7>;
  }
}

// Moments of one triangle against the splines of one leaf box.  The triangle
// is clipped by every interior knot plane, so each piece lies in one knot
// cell per axis and meets (p+1)^3 splines; its spans are found once, at the
// piece's vertex mean.  Each piece's fan triangles take the collapsed Gauss
// rule, and the piece keeps the tile
//   T[i0][i1][c][i2] = sum_q w_q f_c(x_q) N_i0(x_q) N_i1(y_q) N_i2(z_q),
// f_0 = 1 and f_{1+d} = x_d - o_d (o: the triangle's vertex mean), from which
// every RWG and pulse moment of the triangle is a linear combination.
struct PieceTile {
  int span[3];
  double t[8 * 8 * 4 * 8];
};

void triangle_tiles(const LeafKnots& K, const double* tv, const double* o,
                    const std::vector<double>& qx, const std::vector<double>& qw,
                    std::vector<PieceTile>& out) {
  const int p = K.p, sp = K.sp, p1 = p + 1;
  thread_local std::vector<Poly> pieces;
  pieces.resize(1);
  pieces[0].n = 3;
  for (int a = 0; a < 3; ++a)
    for (int d = 0; d < 3; ++d) pieces[0].v[a][d] = tv[3 * a + d];
  Poly L, R;
  for (int axis = 0; axis < 3; ++axis) {
    for (int kk = p + 1; kk < sp; ++kk) {
      const double val = K.U[axis][kk];
      const size_t n0 = pieces.size();
      for (size_t i = 0; i < n0; ++i) {
        const Poly& P = pieces[i];
        double mn = 1e300, mx = -1e300;
        for (int j = 0; j < P.n; ++j) {
          mn = std::min(mn, P.v[j][axis]);
          mx = std::max(mx, P.v[j][axis]);
        }
        if (!(mn < val && val < mx)) continue;
        split(P, axis, val, L, R);
        if (L.n >= 3) {
          pieces[i] = L;
          if (R.n >= 3) pieces.push_back(R);
        } else if (R.n >= 3) {
          pieces[i] = R;
        } else {
          pieces[i].n = 0;  // nothing left of this piece
        }
      }
    }
  }
  const int nq = (int)qx.size();
  const contract_fn contract = contract_for(p1);
  const int W = 4 * p1;
  thread_local std::vector<double> NN, F;
  double N0[8], N1[8], N2[8];
  out.clear();
  for (const Poly& P : pieces) {
    if (P.n < 3) continue;
    double cen[3] = {0, 0, 0};
    for (int i = 0; i < P.n; ++i)
      for (int d = 0; d < 3; ++d) cen[d] += P.v[i][d];
    for (int d = 0; d < 3; ++d) cen[d] /= P.n;
    int span[3];
    for (int d = 0; d < 3; ++d) span[d] = find_span(K.U[d], p, sp, cen[d]);
    double r0[28], r1[28], r2[28];
    span_recip(K.U[0], p, span[0], r0);
    span_recip(K.U[1], p, span[1], r1);
    span_recip(K.U[2], p, span[2], r2);
    const int ld = (P.n - 2) * nq * nq;
    if ((int)NN.size() < p1 * p1 * ld) NN.resize((size_t)p1 * p1 * ld);
    if ((int)F.size() < W * ld) F.resize((size_t)W * ld);
    int Q = 0;
    for (int f = 1; f + 1 < P.n; ++f) {
      const double* A = P.v[0];
      const double* B = P.v[f];
      const double* C = P.v[f + 1];
      double u[3], v[3];
      for (int d = 0; d < 3; ++d) {
        u[d] = B[d] - A[d];
        v[d] = C[d] - A[d];
      }
      double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2],
             cz = u[0] * v[1] - u[1] * v[0];
      double twoa = std::sqrt(cx * cx + cy * cy + cz * cz);
      if (!(twoa > 0)) continue;
      for (int a = 0; a < nq; ++a)
        for (int b = 0; b < nq; ++b, ++Q) {
          double xi = qx[a], eta = qx[b] * (1.0 - qx[a]);
          double w = qw[a] * qw[b] * (1.0 - qx[a]) * twoa;
          double x[3];
          for (int d = 0; d < 3; ++d) x[d] = A[d] + xi * u[d] + eta * v[d];
          basis_nz_r(K.U[0], p, span[0], r0, x[0], N0);
          basis_nz_r(K.U[1], p, span[1], r1, x[1], N1);
          basis_nz_r(K.U[2], p, span[2], r2, x[2], N2);
          for (int i0 = 0; i0 < p1; ++i0)
            for (int i1 = 0; i1 < p1; ++i1) NN[(size_t)(i0 * p1 + i1) * ld + Q] = N0[i0] * N1[i1];
          double* fq = &F[(size_t)Q * W];
          for (int i2 = 0; i2 < p1; ++i2) fq[i2] = w * N2[i2];
          for (int d = 0; d < 3; ++d) {
            const double xd = x[d] - o[d];
            for (int i2 = 0; i2 < p1; ++i2) fq[(1 + d) * p1 + i2] = xd * fq[i2];
          }
        }
    }
    if (Q == 0) continue;
    out.emplace_back();
    PieceTile& T = out.back();
    for (int d = 0; d < 3; ++d) T.span[d] = span[d];
    contract(NN.data(), F.data(), Q, ld, T.t);
  }
}

// block[c][g] += sum_k coef[c][k] T[..][k][..] over the tiles of one triangle
// for a basis function with block origin base and extents ext; ncomp rows of
// coef, each over the 4 tile components.
void scatter_tiles(const std::vector<PieceTile>& tiles, int p, int ncomp, const double* coef,
                   const int* base, const int* ext, double* block) {
  const int p1 = p + 1;
  const int e0 = ext[0], e1 = ext[1], e2 = ext[2];
  const size_t cstride = (size_t)e0 * e1 * e2;
  for (const PieceTile& T : tiles) {
    for (int i0 = 0; i0 < p1; ++i0) {
      const int g0 = T.span[0] - p + i0 - base[0];
      if (g0 < 0 || g0 >= e0) continue;
      for (int i1 = 0; i1 < p1; ++i1) {
        const int g1 = T.span[1] - p + i1 - base[1];
        if (g1 < 0 || g1 >= e1) continue;
        const double* t = T.t + (i0 * p1 + i1) * 4 * p1;
        for (int i2 = 0; i2 < p1; ++i2) {
          const int g2 = T.span[2] - p + i2 - base[2];
          if (g2 < 0 || g2 >= e2) continue;
          const size_t o = ((size_t)g0 * e1 + g1) * e2 + g2;
          for (int c = 0; c < ncomp; ++c) {
            const double* cc = coef + 4 * c;
            block[c * cstride + o] += cc[0] * t[i2] + cc[1] * t[p1 + i2] + cc[2] * t[2 * p1 + i2] +
                                      cc[3] * t[3 * p1 + i2];
          }
        }
      }
    }
  }
}

// Functions sorted by leaf box: sorted RWG i is canonical rwg_perm[i] in leaf
// rwg_box[i] (box_rwg_ptr: CSR over leaves); the same for triangles, with
// tri_rank the inverse of tri_perm.
struct LeafOrder {
  const int32_t *rwg_perm, *rwg_box;
  const int64_t* box_rwg_ptr;
  const int32_t *tri_perm, *tri_box;
  const int64_t* box_tri_ptr;
  const int32_t* tri_rank;
};

// Exact moments (the paper asks only for numerical quadrature; these are exact) of every RWG and pulse in its leaf box's splines
// (knots kcache[leaf], whose s' may differ from leaf to leaf), in sorted
// order: dense blocks over each function's B-spline extents.  One leaf at a
// time: every triangle used by the leaf's RWGs or pulses is integrated once
// against the leaf's splines, and the tiles are combined into each user's
// block; only the leaf's own blocks are written.  with_div adds the RWG
// divergence moments of the direct factorization.
void leaf_moments(const Geometry& g, int p, const std::vector<LeafKnots>& kcache, const LeafOrder& o, bool with_div,
                  MomentBlocks& MR, MomentBlocks& MT, MomentBlocks& MD) {
  const int64_t N = g.N, nt = g.nt;
  const int64_t BD = (int64_t)kcache.size();
  std::vector<double> qx, qw;
  gauss_legendre01((3 * p + 4) / 2, qx, qw);
  auto extents = [&](const LeafKnots& K, const int32_t* verts, int nvv, int* base, int* ext) {
    for (int d = 0; d < 3; ++d) {
      double mn = 1e300, mx = -1e300;
      for (int a = 0; a < nvv; ++a) {
        mn = std::min(mn, g.V[3 * verts[a] + d]);
        mx = std::max(mx, g.V[3 * verts[a] + d]);
      }
      int a0 = find_span(K.U[d], p, K.sp, mn) - p;
      int a1 = find_span(K.U[d], p, K.sp, mx);
      a0 = std::max(a0, 0);
      a1 = std::min(a1, K.sp - 1);
      base[d] = a0;
      ext[d] = a1 - a0 + 1;
    }
  };
  MR.base.assign(3 * N, 0);
  MR.ext.assign(3 * N, 0);
  MR.off.assign(N + 1, 0);
  for (int64_t i = 0; i < N; ++i) {
    int32_t m = o.rwg_perm[i];
    int32_t vv[6];
    for (int a = 0; a < 3; ++a) {
      vv[a] = g.T[3 * g.tri_pm[2 * m] + a];
      vv[3 + a] = g.T[3 * g.tri_pm[2 * m + 1] + a];
    }
    extents(kcache[o.rwg_box[i]], vv, 6, &MR.base[3 * i], &MR.ext[3 * i]);
    MR.off[i + 1] = MR.off[i] + 3LL * MR.ext[3 * i] * MR.ext[3 * i + 1] * MR.ext[3 * i + 2];
  }
  MR.data.assign(MR.off[N], 0.0);
  MT.base.assign(3 * nt, 0);
  MT.ext.assign(3 * nt, 0);
  MT.off.assign(nt + 1, 0);
  for (int64_t i = 0; i < nt; ++i) {
    int32_t t = o.tri_perm[i];
    extents(kcache[o.tri_box[i]], &g.T[3 * t], 3, &MT.base[3 * i], &MT.ext[3 * i]);
    MT.off[i + 1] = MT.off[i] + (int64_t)MT.ext[3 * i] * MT.ext[3 * i + 1] * MT.ext[3 * i + 2];
  }
  MT.data.assign(MT.off[nt], 0.0);
  if (with_div) {
    MD.base = MR.base;
    MD.ext = MR.ext;
    MD.off.assign(N + 1, 0);
    for (int64_t i = 0; i < N; ++i) MD.off[i + 1] = MD.off[i] + (MR.off[i + 1] - MR.off[i]) / 3;
    MD.data.assign(MD.off[N], 0.0);
  }
#pragma omp parallel
  {
    std::vector<PieceTile> tiles;
    std::vector<int32_t> tris;
#pragma omp for schedule(dynamic, 4)
    for (int64_t b = 0; b < BD; ++b) {
      const LeafKnots& K = kcache[b];
      tris.clear();
      for (int64_t i = o.box_rwg_ptr[b]; i < o.box_rwg_ptr[b + 1]; ++i)
        for (int s = 0; s < 2; ++s) tris.push_back(g.tri_pm[2 * o.rwg_perm[i] + s]);
      for (int64_t i = o.box_tri_ptr[b]; i < o.box_tri_ptr[b + 1]; ++i) tris.push_back(o.tri_perm[i]);
      std::sort(tris.begin(), tris.end());
      tris.erase(std::unique(tris.begin(), tris.end()), tris.end());
      for (int32_t t : tris) {
        double tv[9], oc[3] = {0, 0, 0};
        for (int a = 0; a < 3; ++a)
          for (int d = 0; d < 3; ++d) {
            tv[3 * a + d] = g.V[3 * g.T[3 * t + a] + d];
            oc[d] += tv[3 * a + d] / 3.0;
          }
        triangle_tiles(K, tv, oc, qx, qw, tiles);
        // RWGs of the leaf on this triangle: sigma / (2a) (x - x_free)
        for (int64_t i = o.box_rwg_ptr[b]; i < o.box_rwg_ptr[b + 1]; ++i) {
          const int32_t m = o.rwg_perm[i];
          for (int s = 0; s < 2; ++s) {
            if (g.tri_pm[2 * m + s] != t) continue;
            const double* xf = &g.V[3 * g.free_pm[2 * m + s]];
            const double sc = (s == 0 ? 1.0 : -1.0) / (2.0 * g.area[t]);
            double coef[12] = {0};
            for (int d = 0; d < 3; ++d) {
              coef[4 * d] = sc * (oc[d] - xf[d]);
              coef[4 * d + 1 + d] = sc;
            }
            scatter_tiles(tiles, p, 3, coef, &MR.base[3 * i], &MR.ext[3 * i], &MR.data[MR.off[i]]);
            if (with_div) {
              // div f = +-1 / a on c+- (the same sigma / (2a) times 2)
              const double cd[4] = {2.0 * sc, 0, 0, 0};
              scatter_tiles(tiles, p, 1, cd, &MD.base[3 * i], &MD.ext[3 * i], &MD.data[MD.off[i]]);
            }
          }
        }
        // the pulse of this triangle, if it belongs to the leaf: 1 / a
        const int64_t ti = o.tri_rank[t];
        if (o.tri_box[ti] == (int32_t)b) {
          const double coef[4] = {1.0 / g.area[t], 0, 0, 0};
          scatter_tiles(tiles, p, 1, coef, &MT.base[3 * ti], &MT.ext[3 * ti], &MT.data[MT.off[ti]]);
        }
      }
    }
  }
}
}  // namespace

// Interaction lists and translation tiles of every grid level (Sec. III-C):
// pairs of non-adjacent boxes whose parents are adjacent, every non-adjacent
// pair on the top grid level.  Needs the boxes, parents and children.
static void build_translation_lists(Plan& P) {
  const int D = P.D;
  // interaction lists per grid level
  for (int ell = D; ell >= P.top; --ell) {
    Level& L = P.L(ell);
    size_t B = L.code.size();
    std::unordered_map<int64_t, int32_t> off_id;
    std::vector<std::vector<std::pair<int32_t, int64_t>>> lists(B);
    auto key_of = [](int64_t dx, int64_t dy, int64_t dz) {
      return ((dx + (1LL << 20)) << 42) | ((dy + (1LL << 20)) << 21) | (dz + (1LL << 20));
    };
    for (size_t x = 0; x < B; ++x) {
      const int64_t* xi = &L.ijk[3 * x];
      auto consider = [&](int64_t y) {
        const int64_t* yi = &L.ijk[3 * y];
        int64_t dx = xi[0] - yi[0], dy = xi[1] - yi[1], dz = xi[2] - yi[2];
        if (std::max(std::llabs(dx), std::max(std::llabs(dy), std::llabs(dz))) < 2) return;
        lists[x].push_back({(int32_t)y, key_of(dx, dy, dz)});
      };
      if (ell == P.top) {
        for (size_t y = 0; y < B; ++y) consider((int64_t)y);
      } else {
        const Level& U = P.L(ell - 1);
        int64_t pb = L.parent[x];
        const int64_t* pi = &U.ijk[3 * pb];
        int64_t nb = 1LL << (ell - 1);
        for (int a = -1; a <= 1; ++a)
          for (int b = -1; b <= 1; ++b)
            for (int c = -1; c <= 1; ++c) {
              int64_t q[3] = {pi[0] + a, pi[1] + b, pi[2] + c};
              if (q[0] < 0 || q[1] < 0 || q[2] < 0 || q[0] >= nb || q[1] >= nb || q[2] >= nb) continue;
              int64_t qb = find_code(U.code, morton(q[0], q[1], q[2]));
              if (qb < 0) continue;
              for (int64_t y = U.child_ptr[qb]; y < U.child_ptr[qb + 1]; ++y) consider(y);
            }
      }
      std::sort(lists[x].begin(), lists[x].end());
    }
    std::vector<int64_t> keys;
    for (auto& l : lists)
      for (auto& e : l) keys.push_back(e.second);
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    L.offsets.resize(3 * keys.size());
    for (size_t i = 0; i < keys.size(); ++i) {
      off_id[keys[i]] = (int32_t)i;
      L.offsets[3 * i] = (int32_t)((keys[i] >> 42) - (1LL << 20));
      L.offsets[3 * i + 1] = (int32_t)(((keys[i] >> 21) & ((1LL << 21) - 1)) - (1LL << 20));
      L.offsets[3 * i + 2] = (int32_t)((keys[i] & ((1LL << 21) - 1)) - (1LL << 20));
    }
    L.il_ptr.assign(B + 1, 0);
    for (size_t x = 0; x < B; ++x) {
      L.il_ptr[x + 1] = L.il_ptr[x] + (int64_t)lists[x].size();
      for (auto& e : lists[x]) {
        L.il_src.push_back(e.first);
        L.il_off.push_back(off_id[e.second]);
      }
    }
  }
  // translation tiles.  Top grid level: chunks of TILE_TOP consecutive boxes,
  // every box a source.  Lower levels: the children of one parent, whose
  // interaction lists all lie in the children of the parent's neighbours.
  for (int ell = D; ell >= P.top; --ell) {
    Level& L = P.L(ell);
    const int64_t B = (int64_t)L.code.size();
    std::unordered_map<int64_t, int32_t> off_id;
    for (size_t i = 0; i < L.offsets.size() / 3; ++i) {
      int64_t key = (((int64_t)L.offsets[3 * i] + (1LL << 20)) << 42) |
                    (((int64_t)L.offsets[3 * i + 1] + (1LL << 20)) << 21) | ((int64_t)L.offsets[3 * i + 2] + (1LL << 20));
      off_id[key] = (int32_t)i;
    }
    auto add_tile = [&](const std::vector<int32_t>& tg, const std::vector<int32_t>& sr, int tpad) {
      L.tile_tgt_ptr.push_back((int64_t)L.tile_tgt.size());
      L.tile_src_ptr.push_back((int64_t)L.tile_src.size());
      L.tile_kidx_off.push_back((int64_t)L.tile_kidx.size());
      for (int32_t x : tg) L.tile_tgt.push_back(x);
      for (int32_t y : sr) L.tile_src.push_back(y);
      for (int32_t y : sr)
        for (int a = 0; a < tpad; ++a) {
          int32_t id = -1;
          if (a < (int)tg.size()) {
            const int64_t* xi = &L.ijk[3 * tg[a]];
            const int64_t* yi = &L.ijk[3 * y];
            int64_t dx = xi[0] - yi[0], dy = xi[1] - yi[1], dz = xi[2] - yi[2];
            if (std::max(std::llabs(dx), std::max(std::llabs(dy), std::llabs(dz))) >= 2) {
              int64_t key = ((dx + (1LL << 20)) << 42) | ((dy + (1LL << 20)) << 21) | (dz + (1LL << 20));
              auto it = off_id.find(key);
              if (it == off_id.end()) fail(-1, "internal: offset missing from the translation table");
              id = it->second;
            }
          }
          L.tile_kidx.push_back(id);
        }
    };
    if (L.il_src.empty()) {
      // no far pairs on this level
    } else if (ell == P.top) {
      std::vector<int32_t> all(B);
      std::iota(all.begin(), all.end(), 0);
      for (int64_t x0 = 0; x0 < B; x0 += TILE_TOP) {
        std::vector<int32_t> tg;
        for (int64_t x = x0; x < std::min<int64_t>(B, x0 + TILE_TOP); ++x) tg.push_back((int32_t)x);
        int tpad = (int)((tg.size() + TILE_X - 1) / TILE_X) * TILE_X;
        add_tile(tg, all, tpad);
      }
    } else {
      const Level& U = P.L(ell - 1);
      const int64_t nbp = 1LL << (ell - 1);
      for (size_t pb = 0; pb < U.code.size(); ++pb) {
        std::vector<int32_t> tg, sr;
        for (int64_t c = U.child_ptr[pb]; c < U.child_ptr[pb + 1]; ++c) tg.push_back((int32_t)c);
        if (tg.empty()) continue;  // a leaf of a nonuniform tree
        const int64_t* pi = &U.ijk[3 * pb];
        for (int a = -1; a <= 1; ++a)
          for (int b = -1; b <= 1; ++b)
            for (int c = -1; c <= 1; ++c) {
              int64_t q[3] = {pi[0] + a, pi[1] + b, pi[2] + c};
              if (q[0] < 0 || q[1] < 0 || q[2] < 0 || q[0] >= nbp || q[1] >= nbp || q[2] >= nbp) continue;
              int64_t qb = find_code(U.code, morton(q[0], q[1], q[2]));
              if (qb < 0) continue;
              for (int64_t y = U.child_ptr[qb]; y < U.child_ptr[qb + 1]; ++y) sr.push_back((int32_t)y);
            }
        std::sort(sr.begin(), sr.end());
        add_tile(tg, sr, TILE_X);
      }
    }
    L.tile_tgt_ptr.push_back((int64_t)L.tile_tgt.size());
    L.tile_src_ptr.push_back((int64_t)L.tile_src.size());
    L.tile_kidx_off.push_back((int64_t)L.tile_kidx.size());
    // tensor-core tiles below the top grid level (built from the interaction
    // lists; the top level's own tiles already take every box)
    if (ell != P.top && !L.il_src.empty()) {
      std::vector<int32_t> pos(B, -1);
      for (int64_t x0 = 0; x0 < B; x0 += TILE_TOP) {
        const int64_t x1 = std::min<int64_t>(B, x0 + TILE_TOP);
        std::vector<int32_t> sr;
        for (int64_t x = x0; x < x1; ++x)
          for (int64_t e = L.il_ptr[x]; e < L.il_ptr[x + 1]; ++e) sr.push_back(L.il_src[e]);
        std::sort(sr.begin(), sr.end());
        sr.erase(std::unique(sr.begin(), sr.end()), sr.end());
        const int tpad = (int)(((x1 - x0) + TILE_X - 1) / TILE_X) * TILE_X;
        L.tct_tgt_ptr.push_back((int64_t)L.tct_tgt.size());
        L.tct_src_ptr.push_back((int64_t)L.tct_src.size());
        L.tct_kidx_off.push_back((int64_t)L.tct_kidx.size());
        for (int64_t x = x0; x < x1; ++x) L.tct_tgt.push_back((int32_t)x);
        for (size_t j = 0; j < sr.size(); ++j) {
          L.tct_src.push_back(sr[j]);
          pos[sr[j]] = (int32_t)j;
        }
        const size_t k0 = L.tct_kidx.size();
        L.tct_kidx.resize(k0 + sr.size() * (size_t)tpad, -1);
        for (int64_t x = x0; x < x1; ++x)
          for (int64_t e = L.il_ptr[x]; e < L.il_ptr[x + 1]; ++e)
            L.tct_kidx[k0 + (size_t)pos[L.il_src[e]] * tpad + (size_t)(x - x0)] = L.il_off[e];
        for (int32_t y : sr) pos[y] = -1;
      }
      L.tct_tgt_ptr.push_back((int64_t)L.tct_tgt.size());
      L.tct_src_ptr.push_back((int64_t)L.tct_src.size());
      L.tct_kidx_off.push_back((int64_t)L.tct_kidx.size());
    }
  }
}

// Transfer matrices (Sec. IV-B) and DFT-fused projectors of every level.
static void build_level_matrices(Plan& P) {
  const int D = P.D, p = P.p;
  // transfer matrices C^L, C^R (child level ell -> ell-1), lattice units of
  // the child knot spacing (Sec. IV-B)
  for (int ell = D; ell > P.top; --ell) {
    Level& c = P.L(ell);
    const Level& pa = P.L(ell - 1);
    int r = (int)std::lround(pa.delta / c.delta);
    std::vector<double> Up = open_knots(-pa.sb * r, (pa.s - p + pa.sb) * r, pa.sp, p);
    std::vector<double> UcL = open_knots(-c.sb, (c.s - p) + c.sb, c.sp, p);
    std::vector<double> UcR = open_knots((c.s - p) - c.sb, 2 * (c.s - p) + c.sb, c.sp, p);
    int rr, cc;
    c.CL = restriction_matrix(Up, UcL, p, &rr, &cc);
    c.CR = restriction_matrix(Up, UcR, p, &rr, &cc);
  }
  // DFT-fused projector matrices (n = 2 s_hat - 1)
  const double twopi = 2.0 * 3.14159265358979323846;
  for (int ell = D; ell >= P.top; --ell) {
    Level& L = P.L(ell);
    int n = L.nfft, ns = L.shat, sp = L.sp;
    L.Fn.resize((size_t)n * n);
    for (int f = 0; f < n; ++f)
      for (int t = 0; t < n; ++t) {
        long ft = ((long)f * t) % n;
        double ang = -twopi * (double)ft / n;
        L.Fn[(size_t)f * n + t] = cplx(std::cos(ang), std::sin(ang));
      }
    L.Mf.assign((size_t)n * sp, cplx(0, 0));
    for (int f = 0; f < n; ++f)
      for (int i = 0; i < sp; ++i) {
        cplx acc(0, 0);
        for (int t = 0; t < ns; ++t) acc += L.Fn[(size_t)f * n + t] * L.P[(size_t)t * sp + i];
        L.Mf[(size_t)f * sp + i] = acc;
      }
    L.Mb.assign((size_t)sp * n, cplx(0, 0));
    for (int i = 0; i < sp; ++i)
      for (int f = 0; f < n; ++f) {
        cplx acc(0, 0);
        for (int t = 0; t < ns; ++t) acc += L.P[(size_t)t * sp + i] * std::conj(L.Fn[(size_t)f * n + t]);
        L.Mb[(size_t)i * n + f] = acc / (double)n;
      }
  }
}

// Block offsets of the near field over the near lists of the leaves, and the
// triangle sets, local indices and coefficients of the A assembly.
static void build_near_blocks(Plan& P) {
  const int64_t BD = P.n_leaves, N = P.g.N;
  const Geometry& g = P.g;
  const size_t nblk = P.near_src.size();
  P.blkA_off.assign(nblk + 1, 0);
  P.blkV_off.assign(nblk + 1, 0);
  for (int64_t x = 0; x < BD; ++x)
    for (int64_t j = P.near_ptr[x]; j < P.near_ptr[x + 1]; ++j) {
      int32_t y = P.near_src[j];
      int64_t na = (P.box_rwg_ptr[x + 1] - P.box_rwg_ptr[x]) * (P.box_rwg_ptr[y + 1] - P.box_rwg_ptr[y]);
      int64_t nvv = (P.box_tri_ptr[x + 1] - P.box_tri_ptr[x]) * (P.box_tri_ptr[y + 1] - P.box_tri_ptr[y]);
      P.blkA_off[j + 1] = P.blkA_off[j] + na;
      P.blkV_off[j + 1] = P.blkV_off[j] + nvv;
    }
  P.nnzA = P.blkA_off[nblk];
  P.nnzV = P.blkV_off[nblk];
  // triangle sets of RWGs per box, local indices, coefficients sigma/(2a)
  P.tset_ptr.assign(BD + 1, 0);
  P.tset.clear();
  P.rwg_tl.assign(2 * N, 0);
  P.rwg_loc.assign(2 * N, 0);
  P.rwg_coef.assign(2 * N, 0.0);
  for (int64_t b = 0; b < BD; ++b) {
    std::vector<int32_t> ts;
    for (int64_t i = P.box_rwg_ptr[b]; i < P.box_rwg_ptr[b + 1]; ++i)
      for (int s = 0; s < 2; ++s) ts.push_back(g.tri_pm[2 * P.rwg_perm[i] + s]);
    std::sort(ts.begin(), ts.end());
    ts.erase(std::unique(ts.begin(), ts.end()), ts.end());
    for (int64_t i = P.box_rwg_ptr[b]; i < P.box_rwg_ptr[b + 1]; ++i) {
      int32_t m = P.rwg_perm[i];
      for (int s = 0; s < 2; ++s) {
        int32_t t = g.tri_pm[2 * m + s];
        P.rwg_tl[2 * i + s] = (int32_t)(std::lower_bound(ts.begin(), ts.end(), t) - ts.begin());
        int32_t fv = g.free_pm[2 * m + s];
        int loc = 0;
        for (int a = 0; a < 3; ++a)
          if (g.T[3 * t + a] == fv) loc = a;
        P.rwg_loc[2 * i + s] = loc;
        P.rwg_coef[2 * i + s] = (s == 0 ? 1.0 : -1.0) / (2.0 * g.area[t]);
      }
    }
    for (int32_t t : ts) P.tset.push_back(t);
    P.tset_ptr[b + 1] = (int64_t)P.tset.size();
  }
}

// Exact moments of every function in its own leaf, with the splines of the
// leaf's level.
static void build_moments(Plan& P, bool with_div) {
  const int p = P.p;
  const int64_t BD = P.n_leaves;
  // exact moments: collapsed Gauss rule of degree >= 3p+1 per piece
  std::vector<LeafKnots> kcache(BD);
  for (int64_t b = 0; b < BD; ++b) {
    const Level& L = P.L(P.leaf_level[b]);
    const int64_t box = P.leaf_box[b];
    LeafKnots& K = kcache[b];
    K.p = p;
    K.sp = L.sp;
    K.delta = L.delta;
    for (int d = 0; d < 3; ++d) {
      K.lo[d] = P.root_lo[d] + L.ijk[3 * box + d] * L.h - L.sb * L.delta;
      K.U[d] = open_knots(K.lo[d], K.lo[d] + (L.sp - p) * L.delta, L.sp, p);
    }
  }
  LeafOrder ord{P.rwg_perm.data(), P.rwg_box.data(), P.box_rwg_ptr.data(), P.tri_perm.data(), P.tri_box.data(),
                P.box_tri_ptr.data(), P.tri_rank.data()};
  leaf_moments(P.g, p, kcache, ord, with_div, P.mom_rwg, P.mom_tri, P.mom_div);
}

// Leaves of a uniform tree: the boxes of the deepest level, in order.
static void set_uniform_leaves(Plan& P) {
  const int D = P.D;
  Level& LD = P.L(D);
  const int64_t BD = (int64_t)LD.code.size();
  P.adaptive = false;
  P.n_leaves = BD;
  P.leaf_level.assign(BD, D);
  P.leaf_box.resize(BD);
  std::iota(P.leaf_box.begin(), P.leaf_box.end(), (int64_t)0);
  P.level_leaf_ptr.assign(P.lv.size() + 1, 0);
  P.level_leaf_ptr[P.lv.size()] = BD;
  for (auto& L : P.lv) L.leaf.assign(L.code.size(), 0);
  LD.leaf.assign(BD, 1);
  P.rwg_lbox = P.rwg_box;
  P.tri_lbox = P.tri_box;
}

// Index checks of everything the device kernels index with: every box,
// leaf, function, list and tile index in range, every CSR pointer array
// monotone and closed, every moment block inside its leaf's grid.  A planner
// error becomes EfieError here, before any kernel runs.
static void validate_plan(const Plan& P, bool with_moments) {
  auto check = [](bool ok, const char* what) {
    if (!ok) fail(-1, std::string("internal: plan check failed: ") + what);
  };
  auto csr = [&](const std::vector<int64_t>& ptr, size_t rows, size_t nnz, const char* what) {
    check(ptr.size() == rows + 1 && ptr[0] == 0 && (size_t)ptr[rows] == nnz, what);
    for (size_t i = 0; i < rows; ++i) check(ptr[i] <= ptr[i + 1], what);
  };
  const int nlev = (int)P.lv.size();
  check(nlev == P.D - P.top + 1, "level count");
  for (int ell = P.top; ell <= P.D; ++ell) {
    const Level& L = P.L(ell);
    const size_t B = L.code.size();
    check(L.ijk.size() == 3 * B && L.leaf.size() == B && L.parent.size() == B, "box arrays");
    const size_t O = L.offsets.size() / 3;
    check(L.offsets.size() == 3 * O, "offsets");
    if (ell > P.top) {
      const Level& U = P.L(ell - 1);
      for (size_t b = 0; b < B; ++b) check(L.parent[b] >= 0 && (size_t)L.parent[b] < U.code.size(), "parent");
    }
    if (ell < P.D) {
      csr(L.child_ptr, B, P.L(ell + 1).code.size(), "children");
      const Level& C = P.L(ell + 1);
      for (size_t b = 0; b < B; ++b)
        for (int64_t c = L.child_ptr[b]; c < L.child_ptr[b + 1]; ++c) check(C.parent[c] == (int64_t)b, "children");
    }
    csr(L.il_ptr, B, L.il_src.size(), "interaction list");
    check(L.il_off.size() == L.il_src.size(), "interaction list");
    for (size_t e = 0; e < L.il_src.size(); ++e)
      check(L.il_src[e] >= 0 && (size_t)L.il_src[e] < B && L.il_off[e] >= 0 && (size_t)L.il_off[e] < O,
            "interaction list");
    auto tiles = [&](const std::vector<int64_t>& tp, const std::vector<int64_t>& sp_, const std::vector<int64_t>& kp,
                     const std::vector<int32_t>& tg, const std::vector<int32_t>& sr,
                     const std::vector<int32_t>& kx, const char* what) {
      if (tp.empty()) return;
      const size_t nt = tp.size() - 1;
      csr(tp, nt, tg.size(), what);
      csr(sp_, nt, sr.size(), what);
      csr(kp, nt, kx.size(), what);
      for (int32_t x : tg) check(x >= 0 && (size_t)x < B, what);
      for (int32_t y : sr) check(y >= 0 && (size_t)y < B, what);
      for (int32_t o : kx) check(o >= -1 && o < (int64_t)O, what);
      for (size_t t = 0; t < nt; ++t) {
        const int64_t ntg = tp[t + 1] - tp[t], nsr = sp_[t + 1] - sp_[t];
        check(kp[t + 1] - kp[t] >= ntg * nsr, what);
      }
    };
    tiles(L.tile_tgt_ptr, L.tile_src_ptr, L.tile_kidx_off, L.tile_tgt, L.tile_src, L.tile_kidx, "tiles");
    tiles(L.tct_tgt_ptr, L.tct_src_ptr, L.tct_kidx_off, L.tct_tgt, L.tct_src, L.tct_kidx, "tensor-core tiles");
  }
  // leaves
  const int64_t NL = P.n_leaves;
  check((int64_t)P.leaf_level.size() == NL && (int64_t)P.leaf_box.size() == NL, "leaves");
  csr(P.level_leaf_ptr, (size_t)nlev, (size_t)NL, "leaves per level");
  for (int i = 0; i < nlev; ++i) {
    const Level& L = P.lv[i];
    for (int64_t x = P.level_leaf_ptr[i]; x < P.level_leaf_ptr[i + 1]; ++x)
      check(P.leaf_level[x] == P.top + i && P.leaf_box[x] >= 0 && (size_t)P.leaf_box[x] < L.code.size() &&
                L.leaf[P.leaf_box[x]],
            "leaf box");
  }
  // functions sorted by leaf
  auto functions = [&](const std::vector<int32_t>& perm, const std::vector<int32_t>& leaf,
                       const std::vector<int32_t>& lbox, const std::vector<int64_t>& ptr, int64_t n, const char* what) {
    check((int64_t)perm.size() == n && (int64_t)leaf.size() == n && (int64_t)lbox.size() == n, what);
    csr(ptr, (size_t)NL, (size_t)n, what);
    for (int64_t x = 0; x < NL; ++x)
      for (int64_t i = ptr[x]; i < ptr[x + 1]; ++i) check(leaf[i] == x && lbox[i] == P.leaf_box[x], what);
    std::vector<uint8_t> seen(n, 0);
    for (int32_t c : perm) {
      check(c >= 0 && c < n && !seen[c], what);
      seen[c] = 1;
    }
  };
  functions(P.rwg_perm, P.rwg_box, P.rwg_lbox, P.box_rwg_ptr, P.g.N, "RWG order");
  functions(P.tri_perm, P.tri_box, P.tri_lbox, P.box_tri_ptr, P.g.nt, "triangle order");
  // near blocks over the leaves
  csr(P.near_ptr, (size_t)NL, P.near_src.size(), "near lists");
  for (int32_t y : P.near_src) check(y >= 0 && y < NL, "near lists");
  check(P.blkA_off.size() == P.near_src.size() + 1 && P.blkV_off.size() == P.near_src.size() + 1, "near blocks");
  csr(P.tset_ptr, (size_t)NL, P.tset.size(), "triangle sets");
  if (!with_moments) return;
  // moment blocks inside the grid of each function's leaf
  auto blocks = [&](const MomentBlocks& MB, const std::vector<int32_t>& leaf, int ncomp, const char* what) {
    const size_t n = leaf.size();
    check(MB.base.size() == 3 * n && MB.ext.size() == 3 * n && MB.off.size() == n + 1 && MB.off[0] == 0, what);
    for (size_t i = 0; i < n; ++i) {
      const int sp = P.L(P.leaf_level[leaf[i]]).sp;
      int64_t ne = ncomp;
      for (int d = 0; d < 3; ++d) {
        const int b = MB.base[3 * i + d], e = MB.ext[3 * i + d];
        check(b >= 0 && e >= 0 && b + e <= sp, what);
        ne *= e;
      }
      check(MB.off[i + 1] - MB.off[i] == ne, what);
    }
    check((size_t)MB.off[n] == MB.data.size(), what);
  };
  blocks(P.mom_rwg, P.rwg_box, 3, "RWG moments");
  blocks(P.mom_tri, P.tri_box, 1, "pulse moments");
  if (!P.mom_div.off.empty()) blocks(P.mom_div, P.rwg_box, 1, "divergence moments");
}

// ------------------------------------------------------------------ build
void build_plan(Plan& P, const double* xyz, int64_t nv, const int32_t* tri, int64_t nt,
                double k, int p, double grid_spacing, int levels, int n_splines,
                bool with_moments, bool with_div) {
  if (!(k > 0) || !std::isfinite(k)) fail(-1, "wavenumber must be positive");
  if (p < 1 || p > 6) fail(-1, "spline degree p must be in 1..6");
  if (!(grid_spacing > 0)) fail(-1, "grid spacing must be positive");
  build_geometry(P.g, xyz, nv, tri, nt);
  Geometry& g = P.g;
  P.k = k;
  P.p = p;
  const int s0 = n_splines > 0 ? n_splines : p + 4;
  if (s0 <= p) fail(-1, "n_splines must exceed p");
  const double delta = grid_spacing;
  const double h_leaf = (s0 - p) * delta;
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t v = 0; v < nv; ++v)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], g.V[3 * v + d]);
      hi[d] = std::max(hi[d], g.V[3 * v + d]);
    }
  double edge = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
  int D = 0;
  while (h_leaf * (double)(1LL << D) < edge) {
    ++D;
    if (D > 20) fail(-1, "grid spacing too small for the mesh extent");
  }
  if (levels < 1 || levels > D + 1) fail(-1, "levels must be in 1..depth+1 (depth " + std::to_string(D) + ")");
  P.D = D;
  P.top = D - levels + 1;
  P.n_levels = levels;
  P.root_edge = h_leaf * (double)(1LL << D);
  for (int d = 0; d < 3; ++d) P.root_lo[d] = (lo[d] + hi[d]) * 0.5 - P.root_edge * 0.5;
  const double lam = 2.0 * 3.14159265358979323846 / k;

  // leaf boxes of basis functions
  const int64_t N = g.N;
  std::vector<int64_t> rijk(3 * N), tijk(3 * nt);
  for (int64_t m = 0; m < N; ++m) {
    double mid[3];
    for (int d = 0; d < 3; ++d) mid[d] = (g.V[3 * g.edge[2 * m] + d] + g.V[3 * g.edge[2 * m + 1] + d]) * 0.5;
    box_of(P, mid, D, &rijk[3 * m]);
  }
  for (int64_t t = 0; t < nt; ++t) box_of(P, &g.cen[3 * t], D, &tijk[3 * t]);
  // maximum protrusion (Sec. III-B)
  double prot = 0.0;
  auto upd = [&](const int64_t* ijk, const int32_t* verts, int nvv) {
    for (int d = 0; d < 3; ++d) {
      double blo = P.root_lo[d] + ijk[d] * h_leaf;
      double bhi = blo + h_leaf;
      for (int a = 0; a < nvv; ++a) {
        double x = g.V[3 * verts[a] + d];
        prot = std::max(prot, std::max(blo - x, 0.0));
        prot = std::max(prot, std::max(x - bhi, 0.0));
      }
    }
  };
  for (int64_t m = 0; m < N; ++m) {
    int32_t vv[6];
    for (int a = 0; a < 3; ++a) {
      vv[a] = g.T[3 * g.tri_pm[2 * m] + a];
      vv[3 + a] = g.T[3 * g.tri_pm[2 * m + 1] + a];
    }
    upd(&rijk[3 * m], vv, 6);
  }
  for (int64_t t = 0; t < nt; ++t) upd(&tijk[3 * t], &g.T[3 * t], 3);
  const int sb0 = (int)std::ceil(prot / delta);

  // per-level parameters (Sec. IV-C constant s, Sec. IV-D increasing s)
  P.lv.assign(levels, Level());
  {
    int s = s0, sb = sb0;
    double dl = delta;
    for (int ell = D; ell >= P.top; --ell) {
      double h = P.root_edge / (double)(1LL << ell);
      if (ell < D) {
        if (h < 0.5 * lam) {
          sb = (sb + 1) / 2;
          dl = dl * 2.0;
        } else {
          s = 2 * s - p;
        }
      }
      if (2 * sb >= s - p)
        fail(-1, "grid spacing too small for the mesh: " + std::to_string(sb) +
                     " buffer splines leave no gap between far interpolation domains");
      Level& L = P.L(ell);
      L.level = ell;
      L.h = h;
      L.s = s;
      L.sb = sb;
      L.sp = s + 2 * sb;
      L.delta = dl;
      projector(L.sp, p, L.P, &L.shat);
      if (L.shat <= p) fail(-1, "too few splines after stabilization");
      L.Delta = (L.sp - p) * dl / (L.shat - 1);
      L.nfft = 2 * L.shat - 1;
    }
  }
  // occupied boxes per level in Morton order
  {
    std::vector<uint64_t> codes;
    codes.reserve(N + nt);
    for (int64_t m = 0; m < N; ++m) codes.push_back(morton(rijk[3 * m], rijk[3 * m + 1], rijk[3 * m + 2]));
    for (int64_t t = 0; t < nt; ++t) codes.push_back(morton(tijk[3 * t], tijk[3 * t + 1], tijk[3 * t + 2]));
    std::sort(codes.begin(), codes.end());
    codes.erase(std::unique(codes.begin(), codes.end()), codes.end());
    for (int ell = D; ell >= P.top; --ell) {
      Level& L = P.L(ell);
      L.code = codes;
      L.ijk.resize(3 * codes.size());
      for (size_t b = 0; b < codes.size(); ++b) {
        uint64_t c = codes[b];
        int64_t ii[3] = {0, 0, 0};
        for (int bit = 0; bit < 21; ++bit)
          for (int d = 0; d < 3; ++d) ii[d] |= (int64_t)((c >> (3 * bit + d)) & 1) << bit;
        for (int d = 0; d < 3; ++d) L.ijk[3 * b + d] = ii[d];
      }
      for (auto& c : codes) c >>= 3;
      codes.erase(std::unique(codes.begin(), codes.end()), codes.end());
    }
    for (int ell = D; ell >= P.top; --ell) {
      Level& L = P.L(ell);
      size_t B = L.code.size();
      L.parent.assign(B, -1);
      if (ell > P.top) {
        const Level& U = P.L(ell - 1);
        for (size_t b = 0; b < B; ++b) L.parent[b] = find_code(U.code, L.code[b] >> 3);
      }
      if (ell < D) {
        const Level& C = P.L(ell + 1);
        L.child_ptr.assign(B + 1, 0);
        for (size_t c = 0; c < C.code.size(); ++c) L.child_ptr[C.parent[c] + 1]++;
        for (size_t b = 0; b < B; ++b) L.child_ptr[b + 1] += L.child_ptr[b];
      }
    }
  }
  build_translation_lists(P);
  build_level_matrices(P);

  // sorted basis-function order (by leaf box)
  const Level& LD = P.L(D);
  const size_t BD = LD.code.size();
  {
    std::vector<std::pair<int64_t, int32_t>> kk(N);
    for (int64_t m = 0; m < N; ++m)
      kk[m] = {find_code(LD.code, morton(rijk[3 * m], rijk[3 * m + 1], rijk[3 * m + 2])), (int32_t)m};
    std::sort(kk.begin(), kk.end());
    P.rwg_perm.resize(N);
    P.rwg_box.resize(N);
    P.box_rwg_ptr.assign(BD + 1, 0);
    for (int64_t i = 0; i < N; ++i) {
      P.rwg_perm[i] = kk[i].second;
      P.rwg_box[i] = (int32_t)kk[i].first;
      P.box_rwg_ptr[kk[i].first + 1]++;
    }
    for (size_t b = 0; b < BD; ++b) P.box_rwg_ptr[b + 1] += P.box_rwg_ptr[b];
    std::vector<std::pair<int64_t, int32_t>> tt(nt);
    for (int64_t t = 0; t < nt; ++t)
      tt[t] = {find_code(LD.code, morton(tijk[3 * t], tijk[3 * t + 1], tijk[3 * t + 2])), (int32_t)t};
    std::sort(tt.begin(), tt.end());
    P.tri_perm.resize(nt);
    P.tri_box.resize(nt);
    P.tri_rank.resize(nt);
    P.box_tri_ptr.assign(BD + 1, 0);
    for (int64_t i = 0; i < nt; ++i) {
      P.tri_perm[i] = tt[i].second;
      P.tri_box[i] = (int32_t)tt[i].first;
      P.tri_rank[tt[i].second] = (int32_t)i;
      P.box_tri_ptr[tt[i].first + 1]++;
    }
    for (size_t b = 0; b < BD; ++b) P.box_tri_ptr[b + 1] += P.box_tri_ptr[b];
    P.rwg_tri_sorted.resize(2 * N);
    for (int64_t i = 0; i < N; ++i)
      for (int s = 0; s < 2; ++s) P.rwg_tri_sorted[2 * i + s] = P.tri_rank[g.tri_pm[2 * P.rwg_perm[i] + s]];
  }
  // near lists and block offsets
  {
    P.near_ptr.assign(BD + 1, 0);
    P.near_src.clear();
    int64_t nb = 1LL << D;
    for (size_t x = 0; x < BD; ++x) {
      const int64_t* xi = &LD.ijk[3 * x];
      std::vector<int32_t> l;
      for (int a = -1; a <= 1; ++a)
        for (int b = -1; b <= 1; ++b)
          for (int c = -1; c <= 1; ++c) {
            int64_t q[3] = {xi[0] + a, xi[1] + b, xi[2] + c};
            if (q[0] < 0 || q[1] < 0 || q[2] < 0 || q[0] >= nb || q[1] >= nb || q[2] >= nb) continue;
            int64_t y = find_code(LD.code, morton(q[0], q[1], q[2]));
            if (y >= 0) l.push_back((int32_t)y);
          }
      std::sort(l.begin(), l.end());
      for (int32_t y : l) P.near_src.push_back(y);
      P.near_ptr[x + 1] = (int64_t)P.near_src.size();
    }
  }
  set_uniform_leaves(P);
  build_near_blocks(P);
  if (with_moments) build_moments(P, with_div);
  validate_plan(P, with_moments);
}

// ------------------------------------------------------------ nonuniform tree
namespace {
using Key = std::array<int64_t, 3>;
struct KeyHash {
  size_t operator()(const Key& k) const {
    return (size_t)((uint64_t)k[0] * 0x9E3779B97F4A7C15ull ^ (uint64_t)k[1] * 0xC2B2AE3D27D4EB4Full ^
                    (uint64_t)k[2] * 0x165667B19E3779F9ull);
  }
};

// box of a point on a level: floor((x - root_lo) / h), clamped
Key box_key(const double* x, const double* root_lo, double root_edge, int level) {
  const double h = root_edge / (double)(1LL << level);
  const int64_t nmax = (1LL << level) - 1;
  Key k;
  for (int d = 0; d < 3; ++d) {
    int64_t i = (int64_t)std::floor((x[d] - root_lo[d]) / h);
    k[d] = std::min<int64_t>(std::max<int64_t>(i, 0), nmax);
  }
  return k;
}

// largest distance by which the supports [smin, smax] of the listed functions
// leave the boxes of their points on the given level
double protrusion(const std::vector<int32_t>& ids, const std::vector<double>& pt, const std::vector<double>& smin,
                  const std::vector<double>& smax, const double* root_lo, double root_edge, int level) {
  const double h = root_edge / (double)(1LL << level);
  double prot = 0.0;
  for (int32_t i : ids) {
    const Key k = box_key(&pt[3 * i], root_lo, root_edge, level);
    for (int d = 0; d < 3; ++d) {
      const double blo = root_lo[d] + (double)k[d] * h;
      prot = std::max(prot, std::max(blo - smin[3 * i + d], 0.0));
      prot = std::max(prot, std::max(smax[3 * i + d] - (blo + h), 0.0));
    }
  }
  return prot;
}
}  // namespace

void build_adaptive_plan(AdaptivePlan& A, const double* xyz, int64_t nv, const int32_t* tri, int64_t nt,
                         double k, int p, const AdaptiveOptions& o, bool with_moments) {
  if (p < 1 || p > 6) fail(-1, "spline degree p must be in 1..6");
  if (!(k > 0)) fail(-1, "wavenumber must be positive");
  if (o.top < 1) fail(-1, "top grid level must be >= 1");
  Geometry& g = A.g;
  build_geometry(g, xyz, nv, tri, nt);
  A.p = p;
  const int64_t N = g.N;
  // points and support bounds: RWG (edge midpoint, both triangles), triangle (centroid)
  std::vector<double> rpt(3 * N), rmin(3 * N, 1e300), rmax(3 * N, -1e300), tmin(3 * nt, 1e300),
      tmax(3 * nt, -1e300);
  for (int64_t t = 0; t < nt; ++t)
    for (int a = 0; a < 3; ++a)
      for (int d = 0; d < 3; ++d) {
        const double v = g.V[3 * g.T[3 * t + a] + d];
        tmin[3 * t + d] = std::min(tmin[3 * t + d], v);
        tmax[3 * t + d] = std::max(tmax[3 * t + d], v);
      }
  for (int64_t m = 0; m < N; ++m)
    for (int d = 0; d < 3; ++d) {
      rpt[3 * m + d] = (g.V[3 * g.edge[2 * m] + d] + g.V[3 * g.edge[2 * m + 1] + d]) * 0.5;
      for (int s = 0; s < 2; ++s) {
        const int32_t t = g.tri_pm[2 * m + s];
        rmin[3 * m + d] = std::min(rmin[3 * m + d], tmin[3 * t + d]);
        rmax[3 * m + d] = std::max(rmax[3 * m + d], tmax[3 * t + d]);
      }
    }
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t v = 0; v < nv; ++v)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], g.V[3 * v + d]);
      hi[d] = std::max(hi[d], g.V[3 * v + d]);
    }
  A.root_edge = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
  for (int d = 0; d < 3; ++d) A.root_lo[d] = (lo[d] + hi[d]) * 0.5 - A.root_edge * 0.5;
  const double* rl = A.root_lo;
  const double re = A.root_edge;

  // subdivision, level by level
  struct Members {
    std::vector<int32_t> rwg, tri;
  };
  std::vector<std::unordered_map<Key, Members, KeyHash>> boxes(1);
  std::vector<std::vector<Key>> leaves;
  {
    Members all;
    all.rwg.resize(N);
    all.tri.resize(nt);
    std::iota(all.rwg.begin(), all.rwg.end(), 0);
    std::iota(all.tri.begin(), all.tri.end(), 0);
    boxes[0][Key{0, 0, 0}] = std::move(all);
  }
  for (int level = 0; !boxes[level].empty(); ++level) {
    if (level > 60) fail(-1, "tree too deep");
    leaves.emplace_back();
    std::unordered_map<Key, Members, KeyHash> nxt;
    for (auto& kv : boxes[level]) {
      const Members& mb = kv.second;
      bool split = (int64_t)mb.tri.size() > o.max_elems && level < o.max_depth;
      if (split) {
        const double prot = std::max(protrusion(mb.rwg, rpt, rmin, rmax, rl, re, level + 1),
                                     protrusion(mb.tri, g.cen, tmin, tmax, rl, re, level + 1));
        split = prot <= o.max_prot * re / (double)(1LL << (level + 1));
      }
      if (!split) {
        leaves[level].push_back(kv.first);
        continue;
      }
      for (int32_t i : mb.rwg) nxt[box_key(&rpt[3 * i], rl, re, level + 1)].rwg.push_back(i);
      for (int32_t i : mb.tri) nxt[box_key(&g.cen[3 * i], rl, re, level + 1)].tri.push_back(i);
    }
    boxes.push_back(std::move(nxt));
  }
  int D = -1;
  for (int ell = 0; ell < (int)leaves.size(); ++ell)
    if (!leaves[ell].empty()) D = ell;
  for (int ell = 0; ell < std::min(o.top, (int)leaves.size()); ++ell)
    if (!leaves[ell].empty()) fail(-1, "a leaf lies above the top grid level");
  if (o.top > D) fail(-1, "top grid level below the deepest leaf");
  A.D = D;
  A.top = o.top;

  // per-level parameters, deepest level first
  const double lam = 2.0 * M_PI / k;
  const int s_leaf = o.n_splines > 0 ? o.n_splines : p + 4;
  A.lv.assign(D - o.top + 1, AdaptiveLevel());
  A.rwg_level.assign(N, -1);
  A.rwg_box.assign(N, -1);
  A.tri_level.assign(nt, -1);
  A.tri_box.assign(nt, -1);
  int cur_s = s_leaf, cur_sb = 0;
  for (int ell = D; ell >= o.top; --ell) {
    AdaptiveLevel& L = A.lv[ell - o.top];
    L.level = ell;
    L.h = re / (double)(1LL << ell);
    if (ell < D && L.h >= 0.5 * lam) cur_s = 2 * cur_s - p;
    L.delta = L.h / (double)(cur_s - p);
    for (auto& kv : boxes[ell]) L.key.push_back(kv.first);
    std::sort(L.key.begin(), L.key.end());
    const std::vector<Key>& lk = leaves[ell];
    std::unordered_map<Key, int64_t, KeyHash> index;
    for (size_t b = 0; b < L.key.size(); ++b) index[L.key[b]] = (int64_t)b;
    L.leaf.assign(L.key.size(), 0);
    L.n_rwg.assign(L.key.size(), 0);
    L.n_tri.assign(L.key.size(), 0);
    double prot = 0.0;
    for (const Key& key : lk) {
      const Members& mb = boxes[ell].at(key);
      const int64_t b = index.at(key);
      L.leaf[b] = 1;
      L.n_rwg[b] = (int32_t)mb.rwg.size();
      L.n_tri[b] = (int32_t)mb.tri.size();
      L.n_leaf_rwg += (int64_t)mb.rwg.size();
      L.n_leaf_tri += (int64_t)mb.tri.size();
      for (int32_t i : mb.rwg) {
        A.rwg_level[i] = ell;
        A.rwg_box[i] = (int32_t)b;
      }
      for (int32_t i : mb.tri) {
        A.tri_level[i] = ell;
        A.tri_box[i] = (int32_t)b;
      }
      prot = std::max(prot, std::max(protrusion(mb.rwg, rpt, rmin, rmax, rl, re, ell),
                                     protrusion(mb.tri, g.cen, tmin, tmax, rl, re, ell)));
    }
    const int sb_leaves = (int)std::ceil(prot / L.delta);
    if (ell == D)
      cur_sb = sb_leaves;
    else
      cur_sb = std::max(cur_s == A.lv[ell + 1 - o.top].s ? (cur_sb + 1) / 2 : cur_sb, sb_leaves);
    if (2 * cur_sb >= cur_s - p)
      fail(-1, "buffer splines leave no gap between far interpolation domains on level " + std::to_string(ell));
    L.s = cur_s;
    L.sb = cur_sb;
    L.sp = cur_s + 2 * cur_sb;
    L.shat = L.sp - 2 * S_REMOVE[p];
    if (L.shat <= p) fail(-1, "too few splines after stabilization");
  }
  // parents and children
  auto find = [&](int ell, const Key& key) -> int64_t {
    const auto& kk = A.lv[ell - o.top].key;
    auto it = std::lower_bound(kk.begin(), kk.end(), key);
    return (it != kk.end() && *it == key) ? (int64_t)(it - kk.begin()) : -1;
  };
  for (int ell = o.top; ell <= D; ++ell) {
    AdaptiveLevel& L = A.lv[ell - o.top];
    L.parent.assign(L.key.size(), -1);
    if (ell > o.top)
      for (size_t b = 0; b < L.key.size(); ++b)
        L.parent[b] = find(ell - 1, Key{L.key[b][0] >> 1, L.key[b][1] >> 1, L.key[b][2] >> 1});
  }
  for (int ell = o.top; ell <= D; ++ell) {
    AdaptiveLevel& L = A.lv[ell - o.top];
    L.child_ptr.assign(L.key.size() + 1, 0);
    if (ell == D) continue;
    const AdaptiveLevel& C = A.lv[ell + 1 - o.top];
    for (int64_t pb : C.parent) L.child_ptr[pb + 1]++;
    for (size_t b = 0; b < L.key.size(); ++b) L.child_ptr[b + 1] += L.child_ptr[b];
    L.child.resize(C.key.size());
    std::vector<int64_t> fill(L.child_ptr.begin(), L.child_ptr.end() - 1);
    for (size_t c = 0; c < C.key.size(); ++c) L.child[fill[C.parent[c]]++] = (int64_t)c;
  }
  auto adjacent = [](const Key& a, const Key& b) {
    return std::max(std::llabs(a[0] - b[0]), std::max(std::llabs(a[1] - b[1]), std::llabs(a[2] - b[2]))) <= 1;
  };
  // translated pairs: non-adjacent boxes with adjacent parents; every
  // non-adjacent pair on the top level
  for (int ell = o.top; ell <= D; ++ell) {
    AdaptiveLevel& L = A.lv[ell - o.top];
    int64_t n = 0;
    if (ell == o.top) {
      for (size_t x = 0; x < L.key.size(); ++x)
        for (size_t y = 0; y < L.key.size(); ++y)
          if (!adjacent(L.key[x], L.key[y])) ++n;
    } else {
      const AdaptiveLevel& U = A.lv[ell - 1 - o.top];
      for (size_t x = 0; x < L.key.size(); ++x) {
        const Key& pk = U.key[L.parent[x]];
        for (int a = -1; a <= 1; ++a)
          for (int b = -1; b <= 1; ++b)
            for (int c = -1; c <= 1; ++c) {
              const int64_t q = find(ell - 1, Key{pk[0] + a, pk[1] + b, pk[2] + c});
              if (q < 0) continue;
              for (int64_t j = U.child_ptr[q]; j < U.child_ptr[q + 1]; ++j)
                if (!adjacent(L.key[x], L.key[U.child[j]])) ++n;
            }
      }
    }
    L.n_far_pairs = n;
  }
  // leaves of all levels, level by level from the top
  std::vector<std::vector<int64_t>> leaf_of(A.lv.size());
  A.leaf_level.clear();
  A.leaf_box.clear();
  for (int ell = o.top; ell <= D; ++ell) {
    const AdaptiveLevel& L = A.lv[ell - o.top];
    leaf_of[ell - o.top].assign(L.key.size(), -1);
    for (size_t b = 0; b < L.key.size(); ++b)
      if (L.leaf[b]) {
        leaf_of[ell - o.top][b] = (int64_t)A.leaf_level.size();
        A.leaf_level.push_back(ell);
        A.leaf_box.push_back((int64_t)b);
      }
  }
  const int64_t NL = (int64_t)A.leaf_level.size();
  // functions sorted by leaf, then canonical id
  auto sort_by_leaf = [&](const std::vector<int32_t>& lvl, const std::vector<int32_t>& box, int64_t n,
                          std::vector<int32_t>& perm, std::vector<int32_t>& leaf, std::vector<int64_t>& ptr) {
    std::vector<std::pair<int64_t, int32_t>> kk(n);
    for (int64_t i = 0; i < n; ++i) kk[i] = {leaf_of[lvl[i] - o.top][box[i]], (int32_t)i};
    std::sort(kk.begin(), kk.end());
    perm.resize(n);
    leaf.resize(n);
    ptr.assign(NL + 1, 0);
    for (int64_t i = 0; i < n; ++i) {
      perm[i] = kk[i].second;
      leaf[i] = (int32_t)kk[i].first;
      ptr[kk[i].first + 1]++;
    }
    for (int64_t x = 0; x < NL; ++x) ptr[x + 1] += ptr[x];
  };
  sort_by_leaf(A.rwg_level, A.rwg_box, N, A.rwg_perm, A.rwg_leaf, A.leaf_rwg_ptr);
  sort_by_leaf(A.tri_level, A.tri_box, nt, A.tri_perm, A.tri_leaf, A.leaf_tri_ptr);
  A.tri_rank.assign(nt, 0);
  for (int64_t i = 0; i < nt; ++i) A.tri_rank[A.tri_perm[i]] = (int32_t)i;
  // near leaves: x (level lx) and y (level ly) are near when, on the coarser
  // of the two levels, the ancestors are adjacent or equal
  A.near_ptr.assign(NL + 1, 0);
  A.near_src.clear();
  A.near_pairs_rwg = A.near_pairs_tri = 0;
  std::vector<int64_t> stack, ys;
  for (int64_t xl = 0; xl < NL; ++xl) {
    const int lx = A.leaf_level[xl];
    const AdaptiveLevel& LX = A.lv[lx - o.top];
    const Key& kx = LX.key[A.leaf_box[xl]];
    ys.clear();
    // leaves on levels ly <= lx next to (or equal to) x's ancestor
    for (int ly = o.top; ly <= lx; ++ly) {
      const int sh = lx - ly;
      const Key anc{kx[0] >> sh, kx[1] >> sh, kx[2] >> sh};
      for (int a = -1; a <= 1; ++a)
        for (int b = -1; b <= 1; ++b)
          for (int c = -1; c <= 1; ++c) {
            const int64_t y = find(ly, Key{anc[0] + a, anc[1] + b, anc[2] + c});
            if (y >= 0 && leaf_of[ly - o.top][y] >= 0) ys.push_back(leaf_of[ly - o.top][y]);
          }
    }
    // leaves on deeper levels under a box of level lx next to x
    if (lx < D)
      for (int a = -1; a <= 1; ++a)
        for (int b = -1; b <= 1; ++b)
          for (int c = -1; c <= 1; ++c) {
            const int64_t z = find(lx, Key{kx[0] + a, kx[1] + b, kx[2] + c});
            if (z < 0 || LX.leaf[z]) continue;
            // depth-first over the descendants of z: (level, box) packed
            stack.assign(1, ((int64_t)lx << 40) | z);
            while (!stack.empty()) {
              const int64_t e = stack.back();
              stack.pop_back();
              const int le = (int)(e >> 40);
              const int64_t bz = e & ((1LL << 40) - 1);
              const AdaptiveLevel& LE = A.lv[le - o.top];
              for (int64_t j = LE.child_ptr[bz]; j < LE.child_ptr[bz + 1]; ++j) {
                const int64_t cy = LE.child[j];
                const int64_t lid = leaf_of[le + 1 - o.top][cy];
                if (lid >= 0)
                  ys.push_back(lid);
                else
                  stack.push_back(((int64_t)(le + 1) << 40) | cy);
              }
            }
          }
    std::sort(ys.begin(), ys.end());
    for (int64_t y : ys) {
      A.near_src.push_back((int32_t)y);
      A.near_pairs_rwg += (A.leaf_rwg_ptr[xl + 1] - A.leaf_rwg_ptr[xl]) * (A.leaf_rwg_ptr[y + 1] - A.leaf_rwg_ptr[y]);
      A.near_pairs_tri += (A.leaf_tri_ptr[xl + 1] - A.leaf_tri_ptr[xl]) * (A.leaf_tri_ptr[y + 1] - A.leaf_tri_ptr[y]);
    }
    A.near_ptr[xl + 1] = (int64_t)A.near_src.size();
  }
  if (!with_moments) return;
  // exact moments in each function's own leaf, with that level's splines
  std::vector<LeafKnots> kcache(NL);
  for (int64_t x = 0; x < NL; ++x) {
    const AdaptiveLevel& L = A.lv[A.leaf_level[x] - o.top];
    const Key& kx = L.key[A.leaf_box[x]];
    LeafKnots& K = kcache[x];
    K.p = p;
    K.sp = L.sp;
    K.delta = L.delta;
    for (int d = 0; d < 3; ++d) {
      K.lo[d] = A.root_lo[d] + (double)kx[d] * L.h - L.sb * L.delta;
      K.U[d] = open_knots(K.lo[d], K.lo[d] + (L.sp - p) * L.delta, L.sp, p);
    }
  }
  LeafOrder ord{A.rwg_perm.data(), A.rwg_leaf.data(), A.leaf_rwg_ptr.data(), A.tri_perm.data(),
                A.tri_leaf.data(), A.leaf_tri_ptr.data(), A.tri_rank.data()};
  MomentBlocks unused;
  leaf_moments(g, p, kcache, ord, false, A.mom_rwg, A.mom_tri, unused);
}

// The nonuniform tree (Sec. VII) as a plan of the device pipeline: the
// adaptive tree's boxes on every level in Morton order, its per-level spline
// parameters, the translation lists, tiles and matrices of the uniform
// builder, the leaves of all levels as the near field's boxes, and every
// function's moments in its own leaf with that level's splines.
void build_plan_adaptive(Plan& P, const double* xyz, int64_t nv, const int32_t* tri, int64_t nt, double k, int p,
                         const AdaptiveOptions& o, bool with_moments, bool with_div) {
  AdaptivePlan A;
  build_adaptive_plan(A, xyz, nv, tri, nt, k, p, o, false);
  P = Plan();
  P.g = std::move(A.g);
  P.k = k;
  P.p = p;
  P.D = A.D;
  P.top = A.top;
  P.n_levels = A.D - A.top + 1;
  P.root_edge = A.root_edge;
  for (int d = 0; d < 3; ++d) P.root_lo[d] = A.root_lo[d];
  P.adaptive = true;
  const int top = P.top, D = P.D, nlev = P.n_levels;
  P.lv.assign(nlev, Level());
  std::vector<std::vector<int64_t>> newidx(nlev);  // adaptive box index -> Morton position
  for (int ell = top; ell <= D; ++ell) {
    const AdaptiveLevel& AL = A.lv[ell - top];
    Level& L = P.L(ell);
    L.level = ell;
    L.h = AL.h;
    L.s = AL.s;
    L.sb = AL.sb;
    L.sp = AL.sp;
    L.delta = AL.delta;
    projector(L.sp, p, L.P, &L.shat);
    if (L.shat != AL.shat) fail(-1, "internal: stabilized spline count differs from the tree's");
    L.Delta = (L.sp - p) * L.delta / (L.shat - 1);
    L.nfft = 2 * L.shat - 1;
    const size_t B = AL.key.size();
    std::vector<std::pair<uint64_t, int64_t>> cb(B);
    for (size_t b = 0; b < B; ++b) cb[b] = {morton(AL.key[b][0], AL.key[b][1], AL.key[b][2]), (int64_t)b};
    std::sort(cb.begin(), cb.end());
    L.code.resize(B);
    L.ijk.resize(3 * B);
    L.leaf.resize(B);
    newidx[ell - top].resize(B);
    for (size_t b = 0; b < B; ++b) {
      const int64_t a = cb[b].second;
      L.code[b] = cb[b].first;
      for (int d = 0; d < 3; ++d) L.ijk[3 * b + d] = AL.key[a][d];
      L.leaf[b] = AL.leaf[a];
      newidx[ell - top][a] = (int64_t)b;
    }
  }
  for (int ell = D; ell >= top; --ell) {
    Level& L = P.L(ell);
    const size_t B = L.code.size();
    L.parent.assign(B, -1);
    if (ell > top) {
      const Level& U = P.L(ell - 1);
      for (size_t b = 0; b < B; ++b) {
        L.parent[b] = find_code(U.code, L.code[b] >> 3);
        if (L.parent[b] < 0 || U.leaf[L.parent[b]]) fail(-1, "internal: box without an inner parent");
      }
    }
    if (ell < D) {
      const Level& C = P.L(ell + 1);
      L.child_ptr.assign(B + 1, 0);
      for (size_t c = 0; c < C.code.size(); ++c) L.child_ptr[C.parent[c] + 1]++;
      for (size_t b = 0; b < B; ++b) L.child_ptr[b + 1] += L.child_ptr[b];
    }
  }
  // leaves, level by level from the top level
  std::vector<std::vector<int64_t>> leaf_of(nlev);
  P.level_leaf_ptr.assign(nlev + 1, 0);
  for (int ell = top; ell <= D; ++ell) {
    const Level& L = P.L(ell);
    leaf_of[ell - top].assign(L.code.size(), -1);
    for (size_t b = 0; b < L.code.size(); ++b)
      if (L.leaf[b]) {
        leaf_of[ell - top][b] = (int64_t)P.leaf_level.size();
        P.leaf_level.push_back(ell);
        P.leaf_box.push_back((int64_t)b);
      }
    P.level_leaf_ptr[ell - top + 1] = (int64_t)P.leaf_level.size();
  }
  const int64_t NL = (int64_t)P.leaf_level.size();
  P.n_leaves = NL;
  // functions sorted by leaf, then canonical id
  auto sort_by_leaf = [&](const std::vector<int32_t>& lvl, const std::vector<int32_t>& box, int64_t n,
                          std::vector<int32_t>& perm, std::vector<int32_t>& leaf, std::vector<int32_t>& lbox,
                          std::vector<int64_t>& ptr) {
    std::vector<std::pair<int64_t, int32_t>> kk(n);
    for (int64_t i = 0; i < n; ++i) {
      const int e = lvl[i] - top;
      kk[i] = {leaf_of[e][newidx[e][box[i]]], (int32_t)i};
      if (kk[i].first < 0) fail(-1, "internal: function outside a leaf");
    }
    std::sort(kk.begin(), kk.end());
    perm.resize(n);
    leaf.resize(n);
    lbox.resize(n);
    ptr.assign(NL + 1, 0);
    for (int64_t i = 0; i < n; ++i) {
      perm[i] = kk[i].second;
      leaf[i] = (int32_t)kk[i].first;
      lbox[i] = (int32_t)P.leaf_box[kk[i].first];
      ptr[kk[i].first + 1]++;
    }
    for (int64_t x = 0; x < NL; ++x) ptr[x + 1] += ptr[x];
  };
  const int64_t N = P.g.N;
  sort_by_leaf(A.rwg_level, A.rwg_box, N, P.rwg_perm, P.rwg_box, P.rwg_lbox, P.box_rwg_ptr);
  sort_by_leaf(A.tri_level, A.tri_box, nt, P.tri_perm, P.tri_box, P.tri_lbox, P.box_tri_ptr);
  P.tri_rank.assign(nt, 0);
  for (int64_t i = 0; i < nt; ++i) P.tri_rank[P.tri_perm[i]] = (int32_t)i;
  P.rwg_tri_sorted.resize(2 * N);
  for (int64_t i = 0; i < N; ++i)
    for (int s = 0; s < 2; ++s) P.rwg_tri_sorted[2 * i + s] = P.tri_rank[P.g.tri_pm[2 * P.rwg_perm[i] + s]];
  // near leaves of the tree builder, renumbered
  {
    std::vector<int64_t> a2n(NL);
    if ((int64_t)A.leaf_level.size() != NL) fail(-1, "internal: leaf count");
    for (int64_t x = 0; x < NL; ++x) {
      const int e = A.leaf_level[x] - top;
      a2n[x] = leaf_of[e][newidx[e][A.leaf_box[x]]];
    }
    std::vector<std::vector<int32_t>> rows(NL);
    for (int64_t x = 0; x < NL; ++x)
      for (int64_t j = A.near_ptr[x]; j < A.near_ptr[x + 1]; ++j) rows[a2n[x]].push_back((int32_t)a2n[A.near_src[j]]);
    P.near_ptr.assign(NL + 1, 0);
    P.near_src.clear();
    for (int64_t x = 0; x < NL; ++x) {
      std::sort(rows[x].begin(), rows[x].end());
      P.near_src.insert(P.near_src.end(), rows[x].begin(), rows[x].end());
      P.near_ptr[x + 1] = (int64_t)P.near_src.size();
    }
  }
  build_translation_lists(P);
  build_level_matrices(P);
  build_near_blocks(P);
  if (with_moments) build_moments(P, with_div);
  validate_plan(P, with_moments);
}
}  // namespace efie
