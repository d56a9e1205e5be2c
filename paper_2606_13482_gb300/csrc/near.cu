// FP64 near field: triangle-pair Galerkin integrals, block assembly of the
// two near sets of the star factorization (Sec. VI-A: RWG pairs for A and
// triangle pairs for V, each between adjacent leaf boxes), and the blocked
// near-field SpMV.
//
// Quadrature rule (identical in definition to the CPU reference, written
// independently):
//   close pair  |cen_c - cen_c'|^2 < 4 max(emax_c^2, emax_c'^2):
//     outer collapsed 4x4 Gauss rule on c; inner analytic static part
//     int 1/R, int (y-rho)/R over the flat triangle c' (Wilton et al. 1984,
//     Graglia 1993) plus the smooth remainder (exp(-jkR)-1)/(4 pi R) on a 4x4
//     rule; result averaged over the two orientations (c outer / c' outer).
//   regular pair: collapsed 3x3 rule on both triangles.
#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"
#include "device_api.cuh"

namespace efie {

__constant__ double c_q3[3][9];   // xi, eta, w (sum w = 1/2)
__constant__ double c_q4[3][16];

struct TriG {
  double v[3][3];
  double c[3];
  double twoa;
  double emax2;
};

__device__ __forceinline__ void load_tri(const double* __restrict__ V, const int32_t* __restrict__ T,
                                         int t, TriG& g) {
  for (int a = 0; a < 3; ++a) {
    int vi = T[3 * t + a];
    for (int d = 0; d < 3; ++d) g.v[a][d] = V[3 * vi + d];
  }
  double e1[3], e2[3];
  for (int d = 0; d < 3; ++d) {
    g.c[d] = (g.v[0][d] + g.v[1][d] + g.v[2][d]) / 3.0;
    e1[d] = g.v[1][d] - g.v[0][d];
    e2[d] = g.v[2][d] - g.v[0][d];
  }
  double nx = e1[1] * e2[2] - e1[2] * e2[1], ny = e1[2] * e2[0] - e1[0] * e2[2],
         nz = e1[0] * e2[1] - e1[1] * e2[0];
  g.twoa = sqrt(nx * nx + ny * ny + nz * nz);
  double m = 0;
  for (int a = 0; a < 3; ++a) {
    double s = 0;
    for (int d = 0; d < 3; ++d) {
      double t_ = g.v[(a + 1) % 3][d] - g.v[a][d];
      s += t_ * t_;
    }
    m = fmax(m, s);
  }
  g.emax2 = m;
}

__device__ __forceinline__ void rule_point(const TriG& g, double xi, double eta, double* x) {
  for (int d = 0; d < 3; ++d)
    x[d] = g.v[0][d] + xi * (g.v[1][d] - g.v[0][d]) + eta * (g.v[2][d] - g.v[0][d]);
}

#define FOUR_PI 12.566370614359172953850573533118

// ln((R+ + l+)/(R- + l-)) without cancellation
__device__ __forceinline__ double safe_log_ratio(double Rp, double lp, double Rm, double lm,
                                                 double R0sq) {
  double num = lp >= 0 ? Rp + lp : R0sq / fmax(Rp - lp, 1e-300);
  double den = lm >= 0 ? Rm + lm : R0sq / fmax(Rm - lm, 1e-300);
  if (!(num > 0) || !(den > 0)) return 0.0;
  return log(num / den);
}

// Static potentials of triangle g at observation point r:
//   I1 = int 1/|r-r'| dS', Iv = int (r' - rho)/|r-r'| dS', rho = projection of r.
__device__ void static_pot(const TriG& g, const double* r, double& I1, double* Iv, double* rho) {
  double e1[3], e2[3], n[3];
  for (int d = 0; d < 3; ++d) {
    e1[d] = g.v[1][d] - g.v[0][d];
    e2[d] = g.v[2][d] - g.v[0][d];
  }
  n[0] = e1[1] * e2[2] - e1[2] * e2[1];
  n[1] = e1[2] * e2[0] - e1[0] * e2[2];
  n[2] = e1[0] * e2[1] - e1[1] * e2[0];
  double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  for (int d = 0; d < 3; ++d) n[d] /= nn;
  double dh = 0;
  for (int d = 0; d < 3; ++d) dh += (r[d] - g.v[0][d]) * n[d];
  for (int d = 0; d < 3; ++d) rho[d] = r[d] - dh * n[d];
  double ad = fabs(dh);
  I1 = 0.0;
  Iv[0] = Iv[1] = Iv[2] = 0.0;
  for (int i = 0; i < 3; ++i) {
    const double* a = g.v[i];
    const double* b = g.v[(i + 1) % 3];
    double L[3], ll = 0;
    for (int d = 0; d < 3; ++d) {
      L[d] = b[d] - a[d];
      ll += L[d] * L[d];
    }
    ll = sqrt(ll);
    double lh[3] = {L[0] / ll, L[1] / ll, L[2] / ll};
    double uh[3] = {lh[1] * n[2] - lh[2] * n[1], lh[2] * n[0] - lh[0] * n[2],
                    lh[0] * n[1] - lh[1] * n[0]};
    double lm = 0, lp = 0, P0 = 0, Rm = 0, Rp = 0;
    for (int d = 0; d < 3; ++d) {
      lm += (a[d] - rho[d]) * lh[d];
      lp += (b[d] - rho[d]) * lh[d];
      P0 += (a[d] - rho[d]) * uh[d];
      Rm += (r[d] - a[d]) * (r[d] - a[d]);
      Rp += (r[d] - b[d]) * (r[d] - b[d]);
    }
    Rm = sqrt(Rm);
    Rp = sqrt(Rp);
    double R0sq = P0 * P0 + dh * dh;
    double lg = safe_log_ratio(Rp, lp, Rm, lm, R0sq);
    double vterm = 0.5 * (R0sq * lg + lp * Rp - lm * Rm);
    for (int d = 0; d < 3; ++d) Iv[d] += vterm * uh[d];
    if (fabs(P0) > 1e-300) {
      double at = atan2(P0 * lp, R0sq + ad * Rp) - atan2(P0 * lm, R0sq + ad * Rm);
      I1 += P0 * lg - ad * at;
    }
  }
}

// (exp(-jkR) - 1)/(4 pi R), limit -jk/(4 pi) at R = 0
__device__ __forceinline__ double2 smooth_rem(double R, double k) {
  if (!(R > 0)) return make_double2(0.0, -k / FOUR_PI);
  double s, c, sh, ch;
  sincos(k * R, &s, &c);
  sincos(0.5 * k * R, &sh, &ch);
  return make_double2(-2.0 * sh * sh / (FOUR_PI * R), -s / (FOUR_PI * R));
}

__device__ __forceinline__ double2 green(double R, double k) {
  double s, c;
  sincos(k * R, &s, &c);
  double f = 1.0 / (FOUR_PI * R);
  return make_double2(c * f, -s * f);
}

__device__ __forceinline__ bool is_close(const TriG& A, const TriG& B) {
  double d2 = 0;
  for (int d = 0; d < 3; ++d) {
    double t = A.c[d] - B.c[d];
    d2 += t * t;
  }
  return d2 < 4.0 * fmax(A.emax2, B.emax2);
}

// One orientation of the singular rule: outer on A, inner on B.
// Ivv[i][j] = int_A int_B (x - vA_i).(y - vB_j) g ; full = false -> only I0.
__device__ void pair_close_oriented(const TriG& A, const TriG& B, double k, bool full,
                                    double2& I0, double2* Ivv) {
  I0 = make_double2(0, 0);
  if (full)
    for (int q = 0; q < 9; ++q) Ivv[q] = make_double2(0, 0);
  double ya[16][3];
  for (int q = 0; q < 16; ++q) rule_point(B, c_q4[0][q], c_q4[1][q], ya[q]);
  for (int p = 0; p < 16; ++p) {
    double x[3];
    rule_point(A, c_q4[0][p], c_q4[1][p], x);
    double wx = c_q4[2][p] * A.twoa;
    double I1, Iv[3], rho[3];
    static_pot(B, x, I1, Iv, rho);
    double2 in0 = make_double2(I1 / FOUR_PI, 0.0);
    double2 iny[3];
    for (int d = 0; d < 3; ++d) iny[d] = make_double2((Iv[d] + (rho[d] - B.c[d]) * I1) / FOUR_PI, 0.0);
    for (int q = 0; q < 16; ++q) {
      double dd[3], R = 0;
      for (int d = 0; d < 3; ++d) {
        dd[d] = x[d] - ya[q][d];
        R += dd[d] * dd[d];
      }
      R = sqrt(R);
      double2 s = smooth_rem(R, k);
      double wy = c_q4[2][q] * B.twoa;
      s.x *= wy;
      s.y *= wy;
      in0.x += s.x;
      in0.y += s.y;
      if (full)
        for (int d = 0; d < 3; ++d) {
          double yl = ya[q][d] - B.c[d];
          iny[d].x += s.x * yl;
          iny[d].y += s.y * yl;
        }
    }
    I0.x += wx * in0.x;
    I0.y += wx * in0.y;
    if (full) {
      for (int i = 0; i < 3; ++i) {
        double xv[3];
        for (int d = 0; d < 3; ++d) xv[d] = x[d] - A.v[i][d];
        for (int j = 0; j < 3; ++j) {
          double2 acc = make_double2(0, 0);
          for (int d = 0; d < 3; ++d) {
            double bj = B.v[j][d] - B.c[d];
            acc.x += xv[d] * (iny[d].x - bj * in0.x);
            acc.y += xv[d] * (iny[d].y - bj * in0.y);
          }
          Ivv[3 * i + j].x += wx * acc.x;
          Ivv[3 * i + j].y += wx * acc.y;
        }
      }
    }
  }
}

__device__ void pair_regular(const TriG& A, const TriG& B, double k, bool full, double2& I0,
                             double2* Ivv) {
  double ya[9][3], wy[9];
  for (int q = 0; q < 9; ++q) {
    double y[3];
    rule_point(B, c_q3[0][q], c_q3[1][q], y);
    for (int d = 0; d < 3; ++d) ya[q][d] = y[d] - B.c[d];
    wy[q] = c_q3[2][q] * B.twoa;
  }
  double dc[3] = {A.c[0] - B.c[0], A.c[1] - B.c[1], A.c[2] - B.c[2]};
  double2 J00 = make_double2(0, 0), Jx[3], Jy[3], Jxy = make_double2(0, 0);
  for (int d = 0; d < 3; ++d) Jx[d] = Jy[d] = make_double2(0, 0);
  for (int p = 0; p < 9; ++p) {
    double x[3], xl[3];
    rule_point(A, c_q3[0][p], c_q3[1][p], x);
    for (int d = 0; d < 3; ++d) xl[d] = x[d] - A.c[d];
    double wx = c_q3[2][p] * A.twoa;
    double2 S = make_double2(0, 0), Sy[3];
    for (int d = 0; d < 3; ++d) Sy[d] = make_double2(0, 0);
    for (int q = 0; q < 9; ++q) {
      double R = 0;
      for (int d = 0; d < 3; ++d) {
        double t = dc[d] + xl[d] - ya[q][d];
        R += t * t;
      }
      R = sqrt(R);
      double2 g = green(R, k);
      g.x *= wy[q];
      g.y *= wy[q];
      S.x += g.x;
      S.y += g.y;
      if (full)
        for (int d = 0; d < 3; ++d) {
          Sy[d].x += g.x * ya[q][d];
          Sy[d].y += g.y * ya[q][d];
        }
    }
    J00.x += wx * S.x;
    J00.y += wx * S.y;
    if (full)
      for (int d = 0; d < 3; ++d) {
        Jx[d].x += wx * xl[d] * S.x;
        Jx[d].y += wx * xl[d] * S.y;
        Jy[d].x += wx * Sy[d].x;
        Jy[d].y += wx * Sy[d].y;
        Jxy.x += wx * xl[d] * Sy[d].x;
        Jxy.y += wx * xl[d] * Sy[d].y;
      }
  }
  I0 = J00;
  if (!full) return;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double a[3], b[3], ab = 0;
      for (int d = 0; d < 3; ++d) {
        a[d] = A.v[i][d] - A.c[d];
        b[d] = B.v[j][d] - B.c[d];
        ab += a[d] * b[d];
      }
      double2 v = Jxy;
      for (int d = 0; d < 3; ++d) {
        v.x -= a[d] * Jy[d].x + b[d] * Jx[d].x;
        v.y -= a[d] * Jy[d].y + b[d] * Jx[d].y;
      }
      v.x += ab * J00.x;
      v.y += ab * J00.y;
      Ivv[3 * i + j] = v;
    }
}

// Pair integrals of canonical triangles (ta, tb): I0 and (full) Ivv[9].
__device__ void pair_integrals(const double* V, const int32_t* T, int ta, int tb, double k,
                               bool full, double2& I0, double2* Ivv) {
  TriG A, B;
  load_tri(V, T, ta, A);
  load_tri(V, T, tb, B);
  if (!is_close(A, B)) {
    pair_regular(A, B, k, full, I0, Ivv);
    return;
  }
  double2 I0a, I0b, Ia[9], Ib[9];
  pair_close_oriented(A, B, k, full, I0a, Ia);
  pair_close_oriented(B, A, k, full, I0b, Ib);
  I0 = make_double2(0.5 * (I0a.x + I0b.x), 0.5 * (I0a.y + I0b.y));
  if (full)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        Ivv[3 * i + j] = make_double2(0.5 * (Ia[3 * i + j].x + Ib[3 * j + i].x),
                                      0.5 * (Ia[3 * i + j].y + Ib[3 * j + i].y));
}

__device__ __forceinline__ int64_t find_block(const int64_t* off, int64_t n, int64_t e) {
  // largest j with off[j] <= e (off has n+1 entries, off[0] = 0)
  int64_t lo = 0, hi = n;
  while (hi - lo > 1) {
    int64_t mid = (lo + hi) >> 1;
    if (off[mid] <= e) lo = mid; else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------- assembly
// Triangle-pair integrals for the A blocks j in [j0, j1): pair (a, b) of the
// triangle sets T_x x T_y; scratch[e] = {I0, Ivv[9]} (10 double2).
__global__ void k_near_pairs_A(NearDev nd, int64_t j0, int64_t nblk, const int64_t* scr_off,
                               double2* scratch, int64_t total) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  int64_t jl = find_block(scr_off, nblk, e);
  int64_t j = j0 + jl;
  int32_t x = nd.blk_tgt[j], y = nd.near_src[j];
  int64_t ny = nd.tset_ptr[y + 1] - nd.tset_ptr[y];
  int64_t loc = e - scr_off[jl];
  int64_t a = loc / ny, b = loc - a * ny;
  int ta = nd.tset[nd.tset_ptr[x] + a];
  int tb = nd.tset[nd.tset_ptr[y] + b];
  double2 I0, Ivv[9];
  pair_integrals(nd.V, nd.T, ta, tb, nd.k, true, I0, Ivv);
  double2* out = scratch + 10 * e;
  out[0] = I0;
  for (int q = 0; q < 9; ++q) out[1 + q] = Ivv[q];
}

// A block entries from the pair scratch:
// A[i][n] = sum_{s,t} coef_is coef_nt Ivv[(tl_is, tl_nt)][loc_is][loc_nt]
// and, for the direct factorization, the scalar part of the same pair from
// the I0 of the same triangle pairs (div f = sign / area on each side, and
// coef = sign / (2 area)): Phi[i][n] = sum_{s,t} 4 coef_is coef_nt I0
__global__ void k_near_combine_A(NearDev nd, int64_t j0, int64_t nblk, const int64_t* scr_off,
                                 const double2* scratch, int64_t e_begin, int64_t total) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  int64_t eg = e_begin + e;
  int64_t j = find_block(nd.blkA_off + j0, nblk, eg) + j0;
  int32_t x = nd.blk_tgt[j], y = nd.near_src[j];
  if (x > y) return;  // transpose of block (y, x): k_near_mirror
  int64_t nxr = nd.box_rwg_ptr[x + 1] - nd.box_rwg_ptr[x];
  int64_t loc = eg - nd.blkA_off[j];
  int64_t c = loc / nxr, r = loc - c * nxr;  // column-major block
  int64_t i = nd.box_rwg_ptr[x] + r, n = nd.box_rwg_ptr[y] + c;
  int64_t nty = nd.tset_ptr[y + 1] - nd.tset_ptr[y];
  const double2* scr = scratch + 10 * scr_off[j - j0];
  double2 acc = make_double2(0, 0), phi = make_double2(0, 0);
  for (int s = 0; s < 2; ++s)
    for (int t = 0; t < 2; ++t) {
      int64_t pe = (int64_t)nd.rwg_tl[2 * i + s] * nty + nd.rwg_tl[2 * n + t];
      double cf = nd.rwg_coef[2 * i + s] * nd.rwg_coef[2 * n + t];
      double2 v = scr[10 * pe + 1 + 3 * nd.rwg_loc[2 * i + s] + nd.rwg_loc[2 * n + t]];
      acc.x += cf * v.x;
      acc.y += cf * v.y;
      const double2 i0 = scr[10 * pe];
      phi.x += 4.0 * cf * i0.x;
      phi.y += 4.0 * cf * i0.y;
    }
  nd.A[eg] = acc;
  if (nd.Phi) nd.Phi[eg] = phi;
}

// Block (x, y) = transpose of block (y, x).  Block j is column-major
// [ny][nx] (entry (r, c) at c nx + r, r over the functions of x, c over those
// of y); its mirror is [nx][ny], entry (c, r) at r ny + c.  One CTA per listed
// block, 32 x 32 tiles through shared memory so that both the reads and the
// writes are coalesced.
__global__ void __launch_bounds__(256)
k_near_mirror(double2* __restrict__ M, const int64_t* __restrict__ blk_off, const int64_t* __restrict__ box_ptr,
              const int32_t* __restrict__ blk_tgt, const int32_t* __restrict__ near_src,
              const int64_t* __restrict__ mir_blk, const int64_t* __restrict__ mir_src) {
  __shared__ double2 tile[32][33];
  const int64_t j = mir_blk[blockIdx.x], jm = mir_src[blockIdx.x];
  const int32_t x = blk_tgt[j], y = near_src[j];
  const int nx = (int)(box_ptr[x + 1] - box_ptr[x]), ny = (int)(box_ptr[y + 1] - box_ptr[y]);
  double2* dst = M + blk_off[j];
  const double2* src = M + blk_off[jm];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int c0 = 0; c0 < ny; c0 += 32)
    for (int r0 = 0; r0 < nx; r0 += 32) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int r = r0 + ty + 8 * k, c = c0 + tx;
        if (r < nx && c < ny) tile[ty + 8 * k][tx] = src[(int64_t)r * ny + c];
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int c = c0 + ty + 8 * k, r = r0 + tx;
        if (r < nx && c < ny) dst[(int64_t)c * nx + r] = tile[tx][ty + 8 * k];
      }
      __syncthreads();
    }
}

// V entries of a batch of blocks from the A pass's triangle-pair scratch:
// scratch[10 (scr_off[j - j0] + a tl_y + b)] holds I0 of the a-th triangle of
// T_x and the b-th of T_y.  A triangle whose centroid box is x is almost
// always in T_x (it has an RWG in x); where it is not, I0 is computed here.
__global__ void k_near_V_pairs(NearDev nd, int64_t j0, int64_t nblk, const int64_t* scr_off,
                               const double2* scratch, int64_t e_begin, int64_t total) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  int64_t eg = e_begin + e;
  int64_t j = find_block(nd.blkV_off + j0, nblk, eg) + j0;
  int32_t x = nd.blk_tgt[j], y = nd.near_src[j];
  if (x > y) return;  // transpose of block (y, x): k_near_mirror
  int64_t nxt = nd.box_tri_ptr[x + 1] - nd.box_tri_ptr[x];
  int64_t loc = eg - nd.blkV_off[j];
  int64_t b = loc / nxt, a = loc - b * nxt;  // column-major block
  const int64_t ia = nd.box_tri_ptr[x] + a, ib = nd.box_tri_ptr[y] + b;
  const int ta = nd.tri_perm[ia], tb = nd.tri_perm[ib];
  const int32_t la = nd.tri_tl[ia], lb = nd.tri_tl[ib];
  double2 I0;
  if (la >= 0 && lb >= 0) {
    const int64_t nty = nd.tset_ptr[y + 1] - nd.tset_ptr[y];
    I0 = scratch[10 * (scr_off[j - j0] + (int64_t)la * nty + lb)];
  } else {
    double2 dummy[9];
    pair_integrals(nd.V, nd.T, ta, tb, nd.k, false, I0, dummy);
  }
  double sc = 1.0 / (nd.area[ta] * nd.area[tb]);
  nd.Vn[eg] = make_double2(I0.x * sc, I0.y * sc);
}

// ---------------------------------------------------------------- SpMV
// y[r][i] += sum_{blocks} M_blk[row][col] x[r][src_start + col] over the near
// blocks of the target box.  Blocks are column-major ([col][row]), so threads
// that own consecutive rows read one column of a block as one coalesced
// stream; the source box's x values are staged in shared memory, NEAR_CH
// columns at a time, and read as broadcasts.  One CTA per target box; a
// thread owns up to UPT "units" = (row, group of RPT right-hand sides), and
// keeps their sums in registers across all source boxes, so no reduction is
// needed.  Sorted orders; x, y are [nr][n] with leading dimension ld, nr <= 8.
constexpr int NEAR_CH = 128;
constexpr int NEAR_THREADS = 256;

template <int RPT, int UPT>
__global__ void __launch_bounds__(NEAR_THREADS)
k_near_rows(const double2* __restrict__ M, const int64_t* __restrict__ blk_off,
            const int64_t* __restrict__ near_ptr, const int32_t* __restrict__ near_src,
            const int64_t* __restrict__ box_ptr, const double2* __restrict__ x,
            double2* __restrict__ y, int64_t ld, int nr) {
  __shared__ double2 xs[8][NEAR_CH];
  const int xb = blockIdx.x, tid = threadIdx.x;
  const int64_t r0 = box_ptr[xb];
  const int nrow = (int)(box_ptr[xb + 1] - r0);
  const int ngrp = (nr + RPT - 1) / RPT, nunits = nrow * ngrp;
  const int64_t j0 = near_ptr[xb], j1 = near_ptr[xb + 1];
  for (int ubase = 0; ubase < nunits; ubase += UPT * NEAR_THREADS) {
    int row[UPT], grp[UPT];
    bool ok[UPT];
    double2 acc[UPT][RPT];
#pragma unroll
    for (int k = 0; k < UPT; ++k) {
      int u = ubase + k * NEAR_THREADS + tid;
      ok[k] = u < nunits;
      grp[k] = ok[k] ? u / nrow : 0;
      row[k] = ok[k] ? u - grp[k] * nrow : 0;
#pragma unroll
      for (int q = 0; q < RPT; ++q) acc[k][q] = make_double2(0, 0);
    }
    for (int64_t j = j0; j < j1; ++j) {
      const int32_t yb = near_src[j];
      const int64_t c0 = box_ptr[yb];
      const int ncol = (int)(box_ptr[yb + 1] - c0);
      const double2* Mb = M + blk_off[j];
      for (int cb = 0; cb < ncol; cb += NEAR_CH) {
        const int ncc = min(NEAR_CH, ncol - cb);
        __syncthreads();
        for (int i = tid; i < nr * NEAR_CH; i += NEAR_THREADS) {
          int r = i / NEAR_CH, cc = i - r * NEAR_CH;
          if (cc < ncc) xs[r][cc] = x[r * ld + c0 + cb + cc];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < UPT; ++k) {
          if (!ok[k]) continue;
          const double2* Mc = Mb + (int64_t)cb * nrow + row[k];
          for (int cc = 0; cc < ncc; ++cc) {
            double2 a = Mc[(int64_t)cc * nrow];
#pragma unroll
            for (int q = 0; q < RPT; ++q)
              if (grp[k] * RPT + q < nr) cfma(acc[k][q], a, xs[grp[k] * RPT + q][cc]);
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < UPT; ++k) {
      if (!ok[k]) continue;
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        int r = grp[k] * RPT + q;
        if (r >= nr) break;
        double2* yp = y + r * ld + r0 + row[k];
        double2 t = *yp;
        *yp = make_double2(t.x + acc[k][q].x, t.y + acc[k][q].y);
      }
    }
  }
}

// ---------------------------------------------------------------- double-float SpMV
// Mixed form: every FP64 entry a is kept as a pair of floats (a_hi, a_lo) with
// a_hi = fl32(a), a_lo = fl32(a - a_hi) (48-bit significand, same 16 bytes per
// complex entry), and the product runs on the FP32 pipes: a_hi x_hi is formed
// exactly as p + e with one FMA, the cross terms a_hi x_lo + a_lo x_hi are
// added in FP32, and sums use the error-free two-sum, so each row is accurate
// to ~1e-14 relative -- FP64-class results at FP32 instruction rates.

// in place: double2 (re, im) -> float4 (re_hi, re_lo, im_hi, im_lo)
__global__ void k_split_df(double2* __restrict__ a, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double2 v = a[i];
    float rh = (float)v.x, ih = (float)v.y;
    float rl = (float)(v.x - (double)rh), il = (float)(v.y - (double)ih);
    ((float4*)a)[i] = make_float4(rh, rl, ih, il);
  }
}

// out-of-place split of [nr][n] vectors
__global__ void k_split_vec(const double2* __restrict__ x, float4* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double2 v = x[i];
    float rh = (float)v.x, ih = (float)v.y;
    y[i] = make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
  }
}

struct DF {
  float hi, lo;
};
// S += p (error-free two-sum, error folded into lo)
// (the _rn intrinsics are never contracted into FMAs, which would break the
// error-free transformations)
__device__ __forceinline__ void df_add(DF& S, float p) {
  float s = __fadd_rn(S.hi, p);
  float bb = __fsub_rn(s, S.hi);
  float err = __fadd_rn(__fsub_rn(S.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  S.hi = s;
  S.lo = __fadd_rn(S.lo, err);
}

// re/im += a * v for one complex entry a = (re_hi, re_lo, im_hi, im_lo) and
// one complex x value v in the same form.  Each hi x hi product is split into
// p + e exactly by one FMA; e and the hi x lo cross terms go straight into the
// low word, p into the high word by the two-sum.  48 FP32 operations.
__device__ __forceinline__ void df_cmac(DF& re, DF& im, const float4 a, const float4 v) {
  float p1 = __fmul_rn(a.x, v.x), e1 = __fmaf_rn(a.x, v.x, -p1);  // ar xr
  float p2 = __fmul_rn(a.z, v.z), e2 = __fmaf_rn(a.z, v.z, -p2);  // ai xi
  float lr = __fmaf_rn(a.x, v.y, re.lo);
  lr = __fmaf_rn(a.y, v.x, lr);
  lr = __fmaf_rn(-a.z, v.w, lr);
  lr = __fmaf_rn(-a.w, v.z, lr);
  re.lo = __fadd_rn(lr, __fsub_rn(e1, e2));
  df_add(re, p1);
  df_add(re, -p2);
  float p3 = __fmul_rn(a.x, v.z), e3 = __fmaf_rn(a.x, v.z, -p3);  // ar xi
  float p4 = __fmul_rn(a.z, v.x), e4 = __fmaf_rn(a.z, v.x, -p4);  // ai xr
  float li = __fmaf_rn(a.x, v.w, im.lo);
  li = __fmaf_rn(a.y, v.z, li);
  li = __fmaf_rn(a.z, v.y, li);
  li = __fmaf_rn(a.w, v.x, li);
  im.lo = __fadd_rn(li, __fadd_rn(e3, e4));
  df_add(im, p3);
  df_add(im, p4);
}

// Same structure as k_near_rows (column-major blocks, x staged in shared
// memory, sums in registers), in double-float arithmetic.  The next column's
// matrix entry is loaded before the current one is used.
template <int RPT, int UPT>
__global__ void __launch_bounds__(NEAR_THREADS)
k_near_rows_df(const float4* __restrict__ M, const int64_t* __restrict__ blk_off,
               const int64_t* __restrict__ near_ptr, const int32_t* __restrict__ near_src,
               const int64_t* __restrict__ box_ptr, const float4* __restrict__ x,
               double2* __restrict__ y, int64_t ld, int nr, int nch) {
  __shared__ float4 xs[8][NEAR_CH];
  // block = (target box, chunk of 8 right-hand sides), chunks of one box adjacent
  const int xb = blockIdx.x / nch, tid = threadIdx.x;
  x += (int64_t)(blockIdx.x % nch) * 8 * ld;
  y += (int64_t)(blockIdx.x % nch) * 8 * ld;
  const int64_t r0 = box_ptr[xb];
  const int nrow = (int)(box_ptr[xb + 1] - r0);
  const int ngrp = (nr + RPT - 1) / RPT, nunits = nrow * ngrp;
  const int64_t j0 = near_ptr[xb], j1 = near_ptr[xb + 1];
  for (int ubase = 0; ubase < nunits; ubase += UPT * NEAR_THREADS) {
    int row[UPT], grp[UPT];
    bool ok[UPT];
    DF re[UPT][RPT], im[UPT][RPT];
#pragma unroll
    for (int k = 0; k < UPT; ++k) {
      int u = ubase + k * NEAR_THREADS + tid;
      ok[k] = u < nunits;
      grp[k] = ok[k] ? u / nrow : 0;
      row[k] = ok[k] ? u - grp[k] * nrow : 0;
#pragma unroll
      for (int q = 0; q < RPT; ++q) re[k][q] = im[k][q] = DF{0.f, 0.f};
    }
    for (int64_t j = j0; j < j1; ++j) {
      const int32_t yb = near_src[j];
      const int64_t c0 = box_ptr[yb];
      const int ncol = (int)(box_ptr[yb + 1] - c0);
      const float4* Mb = M + blk_off[j];
      for (int cb = 0; cb < ncol; cb += NEAR_CH) {
        const int ncc = min(NEAR_CH, ncol - cb);
        __syncthreads();
        for (int i = tid; i < nr * NEAR_CH; i += NEAR_THREADS) {
          int r = i / NEAR_CH, cc = i - r * NEAR_CH;
          if (cc < ncc) xs[r][cc] = x[r * ld + c0 + cb + cc];
        }
        __syncthreads();
        const float4* Mc[UPT];
        float4 a[UPT];
#pragma unroll
        for (int k = 0; k < UPT; ++k) {
          Mc[k] = Mb + (int64_t)cb * nrow + row[k];
          a[k] = ok[k] ? Mc[k][0] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (int cc = 0; cc < ncc; ++cc) {
          const int cn = cc + 1 < ncc ? cc + 1 : cc;
          float4 an[UPT];
#pragma unroll
          for (int k = 0; k < UPT; ++k) an[k] = ok[k] ? Mc[k][(int64_t)cn * nrow] : a[k];
#pragma unroll
          for (int k = 0; k < UPT; ++k) {
            if (!ok[k]) continue;
#pragma unroll
            for (int q = 0; q < RPT; ++q)
              if (grp[k] * RPT + q < nr) df_cmac(re[k][q], im[k][q], a[k], xs[grp[k] * RPT + q][cc]);
          }
#pragma unroll
          for (int k = 0; k < UPT; ++k) a[k] = an[k];
        }
      }
    }
#pragma unroll
    for (int k = 0; k < UPT; ++k) {
      if (!ok[k]) continue;
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        int r = grp[k] * RPT + q;
        if (r >= nr) break;
        double2* yp = y + r * ld + r0 + row[k];
        double2 t = *yp;
        *yp = make_double2(t.x + ((double)re[k][q].hi + (double)re[k][q].lo),
                           t.y + ((double)im[k][q].hi + (double)im[k][q].lo));
      }
    }
  }
}

// Variant without shared memory and without barriers: each thread reads the
// x values of its right-hand-side group straight from global memory (the
// threads of a group read the same address, one broadcast; a source box's x
// stays in L1 while the block runs over it), so warps never wait for one
// another.  Same units, layouts and arithmetic as k_near_rows_df.
template <int RPT>
__global__ void __launch_bounds__(NEAR_THREADS)
k_near_rows_df_g(const float4* __restrict__ M, const int64_t* __restrict__ blk_off,
                 const int64_t* __restrict__ near_ptr, const int32_t* __restrict__ near_src,
                 const int64_t* __restrict__ box_ptr, const float4* __restrict__ x,
                 double2* __restrict__ y, int64_t ld, int nr, int nch) {
  const int xb = blockIdx.x / nch;
  x += (int64_t)(blockIdx.x % nch) * 8 * ld;
  y += (int64_t)(blockIdx.x % nch) * 8 * ld;
  const int64_t r0 = box_ptr[xb];
  const int nrow = (int)(box_ptr[xb + 1] - r0);
  const int ngrp = (nr + RPT - 1) / RPT, nunits = nrow * ngrp;
  const int64_t j0 = near_ptr[xb], j1 = near_ptr[xb + 1];
  for (int u = threadIdx.x; u < nunits; u += NEAR_THREADS) {
    const int grp = u / nrow, row = u - grp * nrow;
    const int nq = min(RPT, nr - grp * RPT);
    const float4* xg = x + (int64_t)grp * RPT * ld;
    DF re[RPT], im[RPT];
#pragma unroll
    for (int q = 0; q < RPT; ++q) re[q] = im[q] = DF{0.f, 0.f};
    for (int64_t j = j0; j < j1; ++j) {
      const int32_t yb = near_src[j];
      const int64_t c0 = box_ptr[yb];
      const int ncol = (int)(box_ptr[yb + 1] - c0);
      const float4* Mc = M + blk_off[j] + row;
      const float4* xc = xg + c0;
      for (int cc = 0; cc < ncol; ++cc) {
        const float4 a = Mc[(int64_t)cc * nrow];
#pragma unroll
        for (int q = 0; q < RPT; ++q)
          if (q < nq) df_cmac(re[q], im[q], a, xc[q * ld + cc]);
      }
    }
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      if (q >= nq) break;
      double2* yp = y + (grp * RPT + q) * ld + r0 + row;
      double2 t = *yp;
      *yp = make_double2(t.x + ((double)re[q].hi + (double)re[q].lo), t.y + ((double)im[q].hi + (double)im[q].lo));
    }
  }
}

// Full chunks of 8 right-hand sides: one thread per row with all 8 (the
// matrix entry is loaded once for 8 double-float MACs), 128 threads per
// (target box, chunk) block, and the source values staged in shared memory
// 128 columns at a time with 16-byte asynchronous copies, double-buffered:
// the next piece (source box, column block) is in flight while the current
// one is multiplied, so a piece costs two barriers and no exposed load.
constexpr int NDF_T = 128;
constexpr int NDF_CH = 128;
__device__ __forceinline__ void near_cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__global__ void __launch_bounds__(NDF_T)
k_near_rows_df8(const float4* __restrict__ M, const int64_t* __restrict__ blk_off,
                const int64_t* __restrict__ near_ptr, const int32_t* __restrict__ near_src,
                const int64_t* __restrict__ box_ptr, const float4* __restrict__ x, double2* __restrict__ y,
                int64_t ld, int nch) {
  __shared__ __align__(16) float4 xs[2][8][NDF_CH];
  const int xb = blockIdx.x / nch, tid = threadIdx.x;
  x += (int64_t)(blockIdx.x % nch) * 8 * ld;
  y += (int64_t)(blockIdx.x % nch) * 8 * ld;
  const int64_t r0 = box_ptr[xb];
  const int nrow = (int)(box_ptr[xb + 1] - r0);
  const int64_t j0 = near_ptr[xb], j1 = near_ptr[xb + 1];
  for (int ubase = 0; ubase < nrow; ubase += NDF_T) {
    const int row = ubase + tid;
    const bool ok = row < nrow;
    DF re[8], im[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) re[q] = im[q] = DF{0.f, 0.f};
    // pieces (source box j, first column cb) in near-list order; empty boxes skipped
    int64_t ij = j0;
    int icb = 0;
    auto issue = [&](int buf) {
      while (ij < j1 && box_ptr[near_src[ij] + 1] == box_ptr[near_src[ij]]) ++ij;
      if (ij < j1) {
        const int32_t yb = near_src[ij];
        const int64_t c0 = box_ptr[yb];
        const int ncol = (int)(box_ptr[yb + 1] - c0);
        const int ncc = min(NDF_CH, ncol - icb);
        for (int i = tid; i < 8 * ncc; i += NDF_T) {
          const int r = i / ncc, cc = i - r * ncc;
          near_cp16(&xs[buf][r][cc], x + r * ld + c0 + icb + cc);
        }
        icb += NDF_CH;
        if (icb >= ncol) {
          ++ij;
          icb = 0;
        }
      }
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    int64_t cj = j0;
    int ccb = 0, buf = 0;
    issue(0);
    for (;;) {
      while (cj < j1 && box_ptr[near_src[cj] + 1] == box_ptr[near_src[cj]]) ++cj;
      if (cj >= j1) break;
      issue(buf ^ 1);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
      __syncthreads();
      const int32_t yb = near_src[cj];
      const int ncol = (int)(box_ptr[yb + 1] - box_ptr[yb]);
      const int ncc = min(NDF_CH, ncol - ccb);
      if (ok) {
        const float4* Mc = M + blk_off[cj] + (int64_t)ccb * nrow + row;
        float4 a = Mc[0];
        for (int cc = 0; cc < ncc; ++cc) {
          const float4 an = Mc[(int64_t)(cc + 1 < ncc ? cc + 1 : cc) * nrow];
#pragma unroll
          for (int q = 0; q < 8; ++q) df_cmac(re[q], im[q], a, xs[buf][q][cc]);
          a = an;
        }
      }
      __syncthreads();
      ccb += NDF_CH;
      if (ccb >= ncol) {
        ++cj;
        ccb = 0;
      }
      buf ^= 1;
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    if (ok) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        double2* yp = y + q * ld + r0 + row;
        double2 t = *yp;
        *yp = make_double2(t.x + ((double)re[q].hi + (double)re[q].lo), t.y + ((double)im[q].hi + (double)im[q].lo));
      }
    }
    __syncthreads();
  }
}

// The same product with the barriers taken out: a copy warp fills a ring of
// NR_ST shared-memory stages (64 columns x 8 right-hand sides each) with
// 16-byte asynchronous copies, and each of the four row warps waits only for
// the stage it needs (mbarrier "full", 32 copy lanes) and frees it when done
// (mbarrier "empty", one arrival per row warp).  A warp whose rows finish a
// piece early goes on to the next one while the others are still working,
// which a block barrier would not allow.  Every wait is bounded: on a timeout
// the block sets *err, stops, and its outputs are left unwritten.
constexpr int NR_ST = 5;
constexpr int NR_CH = 64;
constexpr long long NR_SPIN = 1LL << 22;
struct NrBar {
  uint64_t full[NR_ST], empty[NR_ST];
  int abort;
};
__device__ __forceinline__ bool nr_wait(uint64_t* b, uint32_t parity, int* abort, int* err) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(b);
  for (long long it = 0; it < NR_SPIN; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 63) == 63 && *reinterpret_cast<volatile int*>(abort)) return false;
  }
  *reinterpret_cast<volatile int*>(abort) = 1;
  if (err) *reinterpret_cast<volatile int*>(err) = 1;
  return false;
}
__global__ void __launch_bounds__(NDF_T + 32)
k_near_rows_df8r(const float4* __restrict__ M, const int64_t* __restrict__ blk_off,
                 const int64_t* __restrict__ near_ptr, const int32_t* __restrict__ near_src,
                 const int64_t* __restrict__ box_ptr, const float4* __restrict__ x, double2* __restrict__ y,
                 int64_t ld, int nch, int* err) {
  __shared__ __align__(16) float4 xs[NR_ST][8][NR_CH];
  __shared__ NrBar bar;
  const int xb = blockIdx.x / nch, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  x += (int64_t)(blockIdx.x % nch) * 8 * ld;
  y += (int64_t)(blockIdx.x % nch) * 8 * ld;
  const int64_t r0 = box_ptr[xb];
  const int nrow = (int)(box_ptr[xb + 1] - r0);
  const int64_t j0 = near_ptr[xb], j1 = near_ptr[xb + 1];
  if (tid == 0) {
    for (int i = 0; i < NR_ST; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"((uint32_t)__cvta_generic_to_shared(&bar.full[i])),
                   "r"(32));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"((uint32_t)__cvta_generic_to_shared(&bar.empty[i])),
                   "r"(NDF_T / 32));
    }
    bar.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  // pieces in near-list order: (source box j, first column cb), empty boxes skipped
  auto next_piece = [&](int64_t& j, int& cb) {
    cb += NR_CH;
    if (cb >= (int)(box_ptr[near_src[j] + 1] - box_ptr[near_src[j]])) {
      ++j;
      cb = 0;
    }
  };
  auto skip_empty = [&](int64_t& j) {
    while (j < j1 && box_ptr[near_src[j] + 1] == box_ptr[near_src[j]]) ++j;
  };
  if (warp == NDF_T / 32) {
    // ------------------------------------------------ copy warp
    uint32_t g = 0;
    bool ok = true;
    for (int ubase = 0; ubase < nrow && ok; ubase += NDF_T) {
      int64_t j = j0;
      int cb = 0;
      for (skip_empty(j); j < j1 && ok; next_piece(j, cb), skip_empty(j), ++g) {
        const int st = (int)(g % NR_ST);
        if (g >= (uint32_t)NR_ST) {
          int w = 1;
          if (lane == 0) w = nr_wait(&bar.empty[st], ((g / NR_ST) - 1) & 1, &bar.abort, err) ? 1 : 0;
          ok = __shfl_sync(0xffffffffu, w, 0) != 0;
          if (!ok) break;
        }
        const int32_t yb = near_src[j];
        const int64_t c0 = box_ptr[yb];
        const int ncc = min(NR_CH, (int)(box_ptr[yb + 1] - c0) - cb);
        for (int i = lane; i < 8 * ncc; i += 32) {
          const int r = i / ncc, cc = i - r * ncc;
          near_cp16(&xs[st][r][cc], x + r * ld + c0 + cb + cc);
        }
        asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(&bar.full[st]))
                     : "memory");
      }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
  } else {
    // ------------------------------------------------ row warps
    uint32_t g = 0;
    bool ok = true;
    for (int ubase = 0; ubase < nrow && ok; ubase += NDF_T) {
      const int row = ubase + tid;
      const bool has = row < nrow;
      DF re[8], im[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) re[q] = im[q] = DF{0.f, 0.f};
      int64_t j = j0;
      int cb = 0;
      for (skip_empty(j); j < j1; next_piece(j, cb), skip_empty(j), ++g) {
        const int st = (int)(g % NR_ST);
        ok = nr_wait(&bar.full[st], (g / NR_ST) & 1, &bar.abort, err);
        if (!ok) break;
        const int32_t yb = near_src[j];
        const int ncc = min(NR_CH, (int)(box_ptr[yb + 1] - box_ptr[yb]) - cb);
        if (has) {
          const float4* Mc = M + blk_off[j] + (int64_t)cb * nrow + row;
          float4 a = Mc[0];
          for (int cc = 0; cc < ncc; ++cc) {
            const float4 an = Mc[(int64_t)(cc + 1 < ncc ? cc + 1 : cc) * nrow];
#pragma unroll
            for (int q = 0; q < 8; ++q) df_cmac(re[q], im[q], a, xs[st][q][cc]);
            a = an;
          }
        }
        __syncwarp();
        if (lane == 0)
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(
                           (uint32_t)__cvta_generic_to_shared(&bar.empty[st]))
                       : "memory");
      }
      if (ok && has) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          double2* yp = y + q * ld + r0 + row;
          double2 t = *yp;
          *yp = make_double2(t.x + ((double)re[q].hi + (double)re[q].lo), t.y + ((double)im[q].hi + (double)im[q].lo));
        }
      }
    }
  }
  __syncthreads();
}

void launch_split_df(double2* a, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  int64_t blocks = ceil_div(n, 256);
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_split_df<<<(unsigned)blocks, 256, 0, s>>>(a, n);
}
void launch_split_vec(const double2* x, float4* y, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  int64_t blocks = ceil_div(n, 256);
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_split_vec<<<(unsigned)blocks, 256, 0, s>>>(x, y, n);
}
// variant 0: full chunks of 8 through k_near_rows_df8, others through
// k_near_rows_df; variant 1: k_near_rows_df_g; variant 2: k_near_rows_df
// only; variant 3: full chunks through k_near_rows_df8r (err: its timeout
// flag).  k_near_rows_df: right-hand sides per unit: all of a 1-, 2- or
// 4-wide chunk; 4 for wider chunks (two units per row, one unit per
// thread).  Full chunks of 8 run in
// one launch of (box, chunk) blocks with the chunks of a box adjacent, so
// the blocks that read one block row of the matrix run together and the
// matrix streams from DRAM about once for all right-hand sides; a last
// partial chunk runs in a launch of its own.
void launch_near_spmv_df(const float4* M, const int64_t* blk_off, const int64_t* near_ptr,
                         const int32_t* near_src, const int64_t* box_ptr, int64_t n_boxes, const float4* x,
                         double2* y, int64_t ld, int nr, int variant, int* err, cudaStream_t s) {
  if (n_boxes <= 0 || nr <= 0) return;
  const int nfull = nr / 8;
  for (int part = 0; part < 2; ++part) {
    const int r0 = part == 0 ? 0 : nfull * 8;
    const int cnt = part == 0 ? 8 : nr - r0;
    const int nch = part == 0 ? nfull : 1;
    if (nch == 0 || cnt == 0) continue;
    const float4* xr = x + (int64_t)r0 * ld;
    double2* yr = y + (int64_t)r0 * ld;
    const unsigned grid = (unsigned)(n_boxes * nch);
    if (variant == 0 && cnt == 8) {
      k_near_rows_df8<<<grid, NDF_T, 0, s>>>(M, blk_off, near_ptr, near_src, box_ptr, xr, yr, ld, nch);
      continue;
    }
    if (variant == 3 && cnt == 8) {
      k_near_rows_df8r<<<grid, NDF_T + 32, 0, s>>>(M, blk_off, near_ptr, near_src, box_ptr, xr, yr, ld, nch, err);
      continue;
    }
    if (variant == 1) {
      if (cnt <= 2)
        k_near_rows_df_g<2><<<grid, NEAR_THREADS, 0, s>>>(M, blk_off, near_ptr, near_src, box_ptr, xr, yr, ld, cnt,
                                                          nch);
      else
        k_near_rows_df_g<4><<<grid, NEAR_THREADS, 0, s>>>(M, blk_off, near_ptr, near_src, box_ptr, xr, yr, ld, cnt,
                                                          nch);
      continue;
    }
    if (cnt == 1)
      k_near_rows_df<1, 1><<<grid, NEAR_THREADS, 0, s>>>(M, blk_off, near_ptr, near_src, box_ptr, xr, yr, ld, cnt,
                                                         nch);
    else if (cnt == 2)
      k_near_rows_df<2, 1><<<grid, NEAR_THREADS, 0, s>>>(M, blk_off, near_ptr, near_src, box_ptr, xr, yr, ld, cnt,
                                                         nch);
    else
      k_near_rows_df<4, 1><<<grid, NEAR_THREADS, 0, s>>>(M, blk_off, near_ptr, near_src, box_ptr, xr, yr, ld, cnt,
                                                         nch);
  }
}

// ---------------------------------------------------------------- launchers
int near_upload_rules(const double* q3, const double* q4) {
  if (cudaMemcpyToSymbol(c_q3, q3, sizeof(double) * 27) != cudaSuccess) return -1;
  if (cudaMemcpyToSymbol(c_q4, q4, sizeof(double) * 48) != cudaSuccess) return -1;
  return 0;
}

void launch_near_pairs_A(const NearDev& nd, int64_t j0, int64_t nblk, const int64_t* scr_off,
                         double2* scratch, int64_t total, cudaStream_t s) {
  if (total <= 0) return;
  k_near_pairs_A<<<(unsigned)ceil_div(total, 128), 128, 0, s>>>(nd, j0, nblk, scr_off, scratch, total);
}
void launch_near_combine_A(const NearDev& nd, int64_t j0, int64_t nblk, const int64_t* scr_off,
                           const double2* scratch, int64_t e_begin, int64_t total, cudaStream_t s) {
  if (total <= 0) return;
  k_near_combine_A<<<(unsigned)ceil_div(total, 256), 256, 0, s>>>(nd, j0, nblk, scr_off, scratch,
                                                                    e_begin, total);
}
void launch_near_V_pairs(const NearDev& nd, int64_t j0, int64_t nblk, const int64_t* scr_off,
                         const double2* scratch, int64_t e_begin, int64_t total, cudaStream_t s) {
  if (total <= 0) return;
  k_near_V_pairs<<<(unsigned)ceil_div(total, 128), 128, 0, s>>>(nd, j0, nblk, scr_off, scratch, e_begin, total);
}
void launch_near_mirror(double2* M, const int64_t* blk_off, const int64_t* box_ptr, const int32_t* blk_tgt,
                        const int32_t* near_src, const int64_t* mir_blk, const int64_t* mir_src, int64_t n,
                        cudaStream_t s) {
  if (n <= 0) return;
  k_near_mirror<<<(unsigned)n, 256, 0, s>>>(M, blk_off, box_ptr, blk_tgt, near_src, mir_blk, mir_src);
}
void launch_near_spmv(const double2* M, const int64_t* blk_off, const int64_t* near_ptr,
                      const int32_t* near_src, const int64_t* box_ptr, int64_t n_boxes,
                      const double2* x, double2* y, int64_t ld, int nr, cudaStream_t s) {
  if (n_boxes <= 0) return;
  for (int r0 = 0; r0 < nr; r0 += 8) {
    int cnt = nr - r0 < 8 ? nr - r0 : 8;
    const double2* xr = x + (int64_t)r0 * ld;
    double2* yr = y + (int64_t)r0 * ld;
    if (cnt == 1)
      k_near_rows<1, 1><<<(unsigned)n_boxes, NEAR_THREADS, 0, s>>>(M, blk_off, near_ptr, near_src, box_ptr, xr,
                                                                    yr, ld, cnt);
    else if (cnt == 2)
      k_near_rows<2, 1><<<(unsigned)n_boxes, NEAR_THREADS, 0, s>>>(M, blk_off, near_ptr, near_src, box_ptr, xr,
                                                                    yr, ld, cnt);
    else
      k_near_rows<4, 1><<<(unsigned)n_boxes, NEAR_THREADS, 0, s>>>(M, blk_off, near_ptr, near_src, box_ptr, xr,
                                                                    yr, ld, cnt);
  }
}

}  // namespace efie
