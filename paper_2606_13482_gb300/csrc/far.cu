// Far-field kernels of the fast matvec (charges through interpolation) and small vector kernels.
//
//  k_anterp : leaf anterpolation q_{d,b} = sum_{n in b} j_n m_{d,n} and the
//             charge component q_{4,b} = sum_{c in b} rho_c m^phi_c
//             (Eq. TAfactor, Sec. VI-A); one CTA per leaf box, one thread
//             per grid point gathering over the moments that cover it.
//  k_mode   : tensor mode products with the knot-insertion transfers
//             C^L / C^R and their transposes (Eq. interleveltransfer, Sec. IV-B).
//  k_dft    : stabilize + zero-pad + DFT fused into one n x s' complex
//             matrix per axis (F P, P = B_stab^{-1} S), inverse likewise
//             (P^T F^{-1}); Sec. III-C, Sec. V-B.
//  k_mac    : frequency-domain translation R_x = sum_{y in IL(x)} K_{x-y} Q_y
//             (Eq. TAfactorBspline, Toeplitz structure), spectra stored
//             frequency-major so one frequency of all boxes is contiguous.
//  k_interp : interpolation (the transpose of anterpolation), one warp per
//             basis function, lanes over channels.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "device_api.cuh"
#include "plan.hpp"
#include "../../include/efie.h"

namespace efie {

// ---------------------------------------------------------------- mode product
template <typename R, bool CM>
__global__ void k_mode(const cpx_t<R>* __restrict__ in, View vin, cpx_t<R>* __restrict__ out,
                       View vout, int64_t B, int C, int ax, int nin, int e0, int e1, int e2,
                       const void* __restrict__ M0, const void* __restrict__ M1,
                       const int8_t* __restrict__ sel, const int64_t* __restrict__ srcmap,
                       bool accumulate) {
  using T = cpx_t<R>;
  const int64_t total = B * e0 * e1 * e2 * (int64_t)C;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t t = idx;
    int c = (int)(t % C);
    t /= C;
    int j2 = (int)(t % e2);
    t /= e2;
    int j1 = (int)(t % e1);
    t /= e1;
    int j0 = (int)(t % e0);
    int64_t b = t / e0;
    int64_t bs = srcmap ? srcmap[b] : b;
    int jo = ax == 0 ? j0 : (ax == 1 ? j1 : j2);
    int64_t step = ax == 0 ? vin.s0 : (ax == 1 ? vin.s1 : vin.s2);
    int64_t base = bs * vin.sb + (int64_t)(ax == 0 ? 0 : j0) * vin.s0 +
                   (int64_t)(ax == 1 ? 0 : j1) * vin.s1 + (int64_t)(ax == 2 ? 0 : j2) * vin.s2 + c;
    const void* Mv = (sel && sel[3 * b + ax]) ? M1 : M0;
    T acc = mk<R>(0, 0);
    if (CM) {
      const T* M = (const T*)Mv + (int64_t)jo * nin;
      for (int i = 0; i < nin; ++i) cfma(acc, M[i], in[base + i * step]);
    } else {
      const R* M = (const R*)Mv + (int64_t)jo * nin;
      for (int i = 0; i < nin; ++i) {
        T v = in[base + i * step];
        acc.x = fma(M[i], v.x, acc.x);
        acc.y = fma(M[i], v.y, acc.y);
      }
    }
    int64_t o = b * vout.sb + (int64_t)j0 * vout.s0 + (int64_t)j1 * vout.s1 + (int64_t)j2 * vout.s2 + c;
    if (accumulate) acc = cadd(acc, out[o]);
    out[o] = acc;
  }
}

// Line form: one thread owns LPT lines (box, the two other indices, LPT
// consecutive channels), loads their nin inputs into registers once and writes
// all nout outputs; the one or two matrices of the pass sit in shared memory,
// so each matrix value read feeds LPT complex MACs.
template <typename R, bool CM, int NMAX, int LPT>
__global__ void k_mode_line(const cpx_t<R>* __restrict__ in, View vin, cpx_t<R>* __restrict__ out,
                            View vout, int64_t B, int C, int ax, int nin, int e0, int e1, int e2,
                            const void* __restrict__ M0, const void* __restrict__ M1,
                            const int8_t* __restrict__ sel, const int64_t* __restrict__ srcmap,
                            bool accumulate) {
  using T = cpx_t<R>;
  extern __shared__ unsigned char smem_raw[];
  const int nout = ax == 0 ? e0 : (ax == 1 ? e1 : e2);
  const int msz = nout * nin;
  const int esz = CM ? (int)sizeof(T) : (int)sizeof(R);
  const int nmat = M1 && M1 != M0 ? 2 : 1;
  for (int i = threadIdx.x; i < msz * esz / 4; i += blockDim.x) {
    ((int*)smem_raw)[i] = ((const int*)M0)[i];
    if (nmat == 2) ((int*)smem_raw)[msz * esz / 4 + i] = ((const int*)M1)[i];
  }
  __syncthreads();
  const int ea = ax == 0 ? e1 : e0, eb = ax == 2 ? e1 : e2;
  const int64_t sa_in = ax == 0 ? vin.s1 : vin.s0, sb_in = ax == 2 ? vin.s1 : vin.s2;
  const int64_t sa_out = ax == 0 ? vout.s1 : vout.s0, sb_out = ax == 2 ? vout.s1 : vout.s2;
  const int64_t step_in = ax == 0 ? vin.s0 : (ax == 1 ? vin.s1 : vin.s2);
  const int64_t step_out = ax == 0 ? vout.s0 : (ax == 1 ? vout.s1 : vout.s2);
  const int CL = C / LPT;  // channel groups
  const int64_t lines = B * ea * eb * (int64_t)CL;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < lines;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t t = idx;
    const int c = (int)(t % CL) * LPT;
    t /= CL;
    const int ib = (int)(t % eb);
    t /= eb;
    const int ia = (int)(t % ea);
    const int64_t b = t / ea;
    const int64_t bs = srcmap ? srcmap[b] : b;
    const T* ip = in + bs * vin.sb + ia * sa_in + ib * sb_in + c;
    T v[NMAX][LPT];
#pragma unroll
    for (int i = 0; i < NMAX; ++i)
      if (i < nin)
#pragma unroll
        for (int l = 0; l < LPT; ++l) v[i][l] = ip[i * step_in + l];
    const unsigned char* Ms = smem_raw + ((nmat == 2 && sel && sel[3 * b + ax]) ? (size_t)msz * esz : 0);
    T* op = out + b * vout.sb + ia * sa_out + ib * sb_out + c;
    for (int j = 0; j < nout; ++j) {
      T acc[LPT];
#pragma unroll
      for (int l = 0; l < LPT; ++l) acc[l] = mk<R>(0, 0);
      if (CM) {
        const T* M = (const T*)Ms + j * nin;
#pragma unroll
        for (int i = 0; i < NMAX; ++i)
          if (i < nin) {
            const T m = M[i];
#pragma unroll
            for (int l = 0; l < LPT; ++l) cfma(acc[l], m, v[i][l]);
          }
      } else {
        const R* M = (const R*)Ms + j * nin;
#pragma unroll
        for (int i = 0; i < NMAX; ++i)
          if (i < nin) {
            const R m = M[i];
#pragma unroll
            for (int l = 0; l < LPT; ++l) {
              acc[l].x = fma(m, v[i][l].x, acc[l].x);
              acc[l].y = fma(m, v[i][l].y, acc[l].y);
            }
          }
      }
#pragma unroll
      for (int l = 0; l < LPT; ++l) {
        T r = acc[l];
        if (accumulate) r = cadd(r, op[j * step_out + l]);
        op[j * step_out + l] = r;
      }
    }
  }
}

template <typename R, bool CM, int NMAX, int LPT>
static void run_mode_line(const cpx_t<R>* in, View vin, cpx_t<R>* out, View vout, int64_t B, int C, int ax,
                          int nin, int e0, int e1, int e2, const void* M0, const void* M1, const int8_t* sel,
                          const int64_t* srcmap, bool accumulate, size_t smem, cudaStream_t s) {
  static SmemAttr attr;
  smem_attr_once(k_mode_line<R, CM, NMAX, LPT>, 96 * 1024, attr.v);
  const int ea = ax == 0 ? e1 : e0, eb = ax == 2 ? e1 : e2;
  int64_t lines = B * ea * eb * (int64_t)(C / LPT);
  int64_t blocks = ceil_div(lines, 128);
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_mode_line<R, CM, NMAX, LPT><<<(unsigned)blocks, 128, smem, s>>>(in, vin, out, vout, B, C, ax, nin, e0, e1, e2,
                                                                     M0, M1, sel, srcmap, accumulate);
}

template <typename R, bool CM>
static bool dispatch_mode_line(const cpx_t<R>* in, View vin, cpx_t<R>* out, View vout, int64_t B, int C, int ax,
                               int nin, int e0, int e1, int e2, const void* M0, const void* M1,
                               const int8_t* sel, const int64_t* srcmap, bool accumulate, size_t smem,
                               cudaStream_t s) {
  const bool two = (C % 2) == 0 && sizeof(R) == 4;
#define EFIE_ML(NM)                                                                                          \
  if (nin <= NM) {                                                                                           \
    if constexpr (sizeof(R) == 4 && NM <= 21) {                                                              \
      if (two) {                                                                                             \
        run_mode_line<R, CM, NM, 2>(in, vin, out, vout, B, C, ax, nin, e0, e1, e2, M0, M1, sel, srcmap,     \
                                    accumulate, smem, s);                                                    \
        return true;                                                                                         \
      }                                                                                                      \
    }                                                                                                        \
    run_mode_line<R, CM, NM, 1>(in, vin, out, vout, B, C, ax, nin, e0, e1, e2, M0, M1, sel, srcmap,         \
                                accumulate, smem, s);                                                        \
    return true;                                                                                             \
  }
  EFIE_ML(9)
  EFIE_ML(13)
  EFIE_ML(21)
  EFIE_ML(40)
#undef EFIE_ML
  return false;
}

// ---------------------------------------------------------------- sibling-shared transfers
// Upward transfer as a tree over the children of each parent: the product
// q_P = sum_c (C_x(c) (x) C_y(c) (x) C_z(c)) q_c is taken one axis at a time,
// summing after each axis the (at most two) partial results that will see the
// same matrices on the remaining axes -- z for children sharing (b_x, b_y),
// then y for groups sharing b_x, then x.  Each output unit g of a pass is
// out[g] = M(bit0[g]) in[src0[g]] + M(bit1[g]) in[src1[g]] (src1 < 0: absent),
// M(0) = C^L, M(1) = C^R, real, applied along axis ax.  The intermediates are
// about a quarter of those of transferring every child separately.
template <typename R, int NMAX, int LPT>
__global__ void k_mode_pair(const cpx_t<R>* __restrict__ in, View vin, cpx_t<R>* __restrict__ out, View vout,
                            int64_t G, int C, int ax, int nin, int e0, int e1, int e2, const R* __restrict__ M0,
                            const R* __restrict__ M1, const int64_t* __restrict__ src0,
                            const int64_t* __restrict__ src1, const int8_t* __restrict__ bit0,
                            const int8_t* __restrict__ bit1) {
  using T = cpx_t<R>;
  extern __shared__ unsigned char smem_raw[];
  const int nout = ax == 0 ? e0 : (ax == 1 ? e1 : e2);
  const int msz = nout * nin;
  R* Ms = reinterpret_cast<R*>(smem_raw);  // [2][nout][nin]
  for (int i = threadIdx.x; i < msz; i += blockDim.x) {
    Ms[i] = M0[i];
    Ms[msz + i] = M1[i];
  }
  __syncthreads();
  const int ea = ax == 0 ? e1 : e0, eb = ax == 2 ? e1 : e2;
  const int64_t sa_in = ax == 0 ? vin.s1 : vin.s0, sb_in = ax == 2 ? vin.s1 : vin.s2;
  const int64_t sa_out = ax == 0 ? vout.s1 : vout.s0, sb_out = ax == 2 ? vout.s1 : vout.s2;
  const int64_t step_in = ax == 0 ? vin.s0 : (ax == 1 ? vin.s1 : vin.s2);
  const int64_t step_out = ax == 0 ? vout.s0 : (ax == 1 ? vout.s1 : vout.s2);
  const int CL = C / LPT;
  const int64_t lines = G * ea * eb * (int64_t)CL;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < lines;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t t = idx;
    const int c = (int)(t % CL) * LPT;
    t /= CL;
    const int ib = (int)(t % eb);
    t /= eb;
    const int ia = (int)(t % ea);
    const int64_t g = t / ea;
    // g0 < 0: an output without inputs (a leaf on the parent level of a
    // nonuniform tree), written as zeros
    const int64_t g0 = src0[g], g1 = src1[g];
    const T* ip0 = in + (g0 >= 0 ? g0 : 0) * vin.sb + ia * sa_in + ib * sb_in + c;
    const T* ip1 = in + (g1 >= 0 ? g1 : (g0 >= 0 ? g0 : 0)) * vin.sb + ia * sa_in + ib * sb_in + c;
    T v0[NMAX][LPT], v1[NMAX][LPT];
#pragma unroll
    for (int i = 0; i < NMAX; ++i)
      if (i < nin)
#pragma unroll
        for (int l = 0; l < LPT; ++l) {
          v0[i][l] = g0 >= 0 ? ip0[i * step_in + l] : mk<R>(0, 0);
          v1[i][l] = g1 >= 0 ? ip1[i * step_in + l] : mk<R>(0, 0);
        }
    const R* Ma = Ms + (bit0[g] ? msz : 0);
    const R* Mb = Ms + (g1 >= 0 && bit1[g] ? msz : 0);
    T* op = out + g * vout.sb + ia * sa_out + ib * sb_out + c;
    for (int j = 0; j < nout; ++j) {
      T acc[LPT];
#pragma unroll
      for (int l = 0; l < LPT; ++l) acc[l] = mk<R>(0, 0);
#pragma unroll
      for (int i = 0; i < NMAX; ++i)
        if (i < nin) {
          const R ma = Ma[j * nin + i], mb = Mb[j * nin + i];
#pragma unroll
          for (int l = 0; l < LPT; ++l) {
            acc[l].x = fma(ma, v0[i][l].x, acc[l].x);
            acc[l].y = fma(ma, v0[i][l].y, acc[l].y);
            acc[l].x = fma(mb, v1[i][l].x, acc[l].x);
            acc[l].y = fma(mb, v1[i][l].y, acc[l].y);
          }
        }
#pragma unroll
      for (int l = 0; l < LPT; ++l) op[j * step_out + l] = acc[l];
    }
  }
}

template <typename R>
void launch_mode_pair(const cpx_t<R>* in, View vin, cpx_t<R>* out, View vout, int64_t G, int C, int ax, int nin,
                      int e0, int e1, int e2, const R* M0, const R* M1, const int64_t* src0, const int64_t* src1,
                      const int8_t* bit0, const int8_t* bit1, cudaStream_t s) {
  const int ea = ax == 0 ? e1 : e0, eb = ax == 2 ? e1 : e2;
  const int nout = ax == 0 ? e0 : (ax == 1 ? e1 : e2);
  if (G <= 0) return;
  const size_t smem = 2 * sizeof(R) * (size_t)nout * nin;
  const bool two = (C % 2) == 0 && sizeof(R) == 4;
  const int lpt = two ? 2 : 1;
  const int64_t lines = G * ea * eb * (int64_t)(C / lpt);
  int64_t blocks = ceil_div(lines, 128);
  if (blocks > 152 * 32) blocks = 152 * 32;
#define EFIE_MP(NM)                                                                                          \
  if (nin <= NM) {                                                                                           \
    if (two && NM <= 9) {                                                                                    \
      auto k = k_mode_pair<R, NM, (sizeof(R) == 4 && NM <= 9) ? 2 : 1>;                                      \
      k<<<(unsigned)blocks, 128, smem, s>>>(in, vin, out, vout, G, C, ax, nin, e0, e1, e2, M0, M1, src0,    \
                                            src1, bit0, bit1);                                               \
    } else {                                                                                                 \
      const int64_t lines1 = G * ea * eb * (int64_t)C;                                                       \
      int64_t blocks1 = ceil_div(lines1, 128);                                                               \
      if (blocks1 > 152 * 32) blocks1 = 152 * 32;                                                            \
      auto k = k_mode_pair<R, NM, 1>;                                                                        \
      k<<<(unsigned)blocks1, 128, smem, s>>>(in, vin, out, vout, G, C, ax, nin, e0, e1, e2, M0, M1, src0,   \
                                             src1, bit0, bit1);                                              \
    }                                                                                                        \
    return;                                                                                                  \
  }
  EFIE_MP(9)
  EFIE_MP(13)
  EFIE_MP(21)
  EFIE_MP(TRANSFER_MAX_SPLINES)
#undef EFIE_MP
  throw EfieError{EFIE_EINVAL, "transfer: more than 40 splines per axis below the top level"};
}

// ---------------------------------------------------------------- DFT passes
// The transform passes apply M = F P (forward, n x s') or M = P^T F^{-1}
// (inverse, s' x n) along one axis, F the n-point DFT and P real.  Because F's
// rows f and n - f (columns, for F^{-1}) are complex conjugates and P is real,
// M[n-f] = conj(M[f]) (forward) and M[:, n-f] = conj(M[:, f]) (inverse), so a
// pair of outputs (inputs) shares one set of real products:
//   forward: with M[f] = A + iB and four real sums S1 = sum A Re v,
//            S2 = sum B Im v, S3 = sum A Im v, S4 = sum B Re v,
//            y_f = (S1 - S2) + i (S3 + S4), y_{n-f} = (S1 + S2) + i (S3 - S4);
//   inverse: M v_f + conj(M) v_{n-f} = A u + i B w with u = v_f + v_{n-f},
//            w = v_f - v_{n-f}.
// That is half the multiply-adds of the dense product, with only rows
// (columns) 0 .. n/2 of M read.  Same line mapping as k_mode_line.
template <typename R, int NMAX, int LPT>
__global__ void k_dft_fwd_line(const cpx_t<R>* __restrict__ in, View vin, cpx_t<R>* __restrict__ out, View vout,
                               int64_t B, int C, int ax, int nin, int e0, int e1, int e2,
                               const cpx_t<R>* __restrict__ M, int n) {
  using T = cpx_t<R>;
  extern __shared__ unsigned char smem_raw[];
  T* Ms = reinterpret_cast<T*>(smem_raw);  // rows 0 .. n/2 of M
  const int nh = n / 2 + 1;
  for (int i = threadIdx.x; i < nh * nin; i += blockDim.x) Ms[i] = M[i];
  __syncthreads();
  const int ea = ax == 0 ? e1 : e0, eb = ax == 2 ? e1 : e2;
  const int64_t sa_in = ax == 0 ? vin.s1 : vin.s0, sb_in = ax == 2 ? vin.s1 : vin.s2;
  const int64_t sa_out = ax == 0 ? vout.s1 : vout.s0, sb_out = ax == 2 ? vout.s1 : vout.s2;
  const int64_t step_in = ax == 0 ? vin.s0 : (ax == 1 ? vin.s1 : vin.s2);
  const int64_t step_out = ax == 0 ? vout.s0 : (ax == 1 ? vout.s1 : vout.s2);
  const int CL = C / LPT;
  const int64_t lines = B * ea * eb * (int64_t)CL;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < lines;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t t = idx;
    const int c = (int)(t % CL) * LPT;
    t /= CL;
    const int ib = (int)(t % eb);
    t /= eb;
    const int ia = (int)(t % ea);
    const int64_t b = t / ea;
    const T* ip = in + b * vin.sb + ia * sa_in + ib * sb_in + c;
    T v[NMAX][LPT];
#pragma unroll
    for (int i = 0; i < NMAX; ++i)
      if (i < nin)
#pragma unroll
        for (int l = 0; l < LPT; ++l) v[i][l] = ip[i * step_in + l];
    T* op = out + b * vout.sb + ia * sa_out + ib * sb_out + c;
    for (int f = 0; f < nh; ++f) {
      R s1[LPT], s2[LPT], s3[LPT], s4[LPT];
#pragma unroll
      for (int l = 0; l < LPT; ++l) s1[l] = s2[l] = s3[l] = s4[l] = (R)0;
      const T* Mr = Ms + f * nin;
#pragma unroll
      for (int i = 0; i < NMAX; ++i)
        if (i < nin) {
          const T m = Mr[i];
#pragma unroll
          for (int l = 0; l < LPT; ++l) {
            s1[l] = fma(m.x, v[i][l].x, s1[l]);
            s2[l] = fma(m.y, v[i][l].y, s2[l]);
            s3[l] = fma(m.x, v[i][l].y, s3[l]);
            s4[l] = fma(m.y, v[i][l].x, s4[l]);
          }
        }
      const bool pair = f != 0 && 2 * f != n;
#pragma unroll
      for (int l = 0; l < LPT; ++l) {
        op[f * step_out + l] = mk<R>(s1[l] - s2[l], s3[l] + s4[l]);
        if (pair) op[(n - f) * step_out + l] = mk<R>(s1[l] + s2[l], s3[l] - s4[l]);
      }
    }
  }
}

// Inverse passes keep the nout (= s') outputs of a line in registers and
// stream the conjugate input pairs (f, n - f) through them.
template <typename R, int AMAX, int LPT>
__global__ void k_dft_inv_line(const cpx_t<R>* __restrict__ in, View vin, cpx_t<R>* __restrict__ out, View vout,
                               int64_t B, int C, int ax, int nin_unused, int e0, int e1, int e2,
                               const cpx_t<R>* __restrict__ M, int n) {
  using T = cpx_t<R>;
  extern __shared__ unsigned char smem_raw[];
  T* Ms = reinterpret_cast<T*>(smem_raw);  // [f][a], f = 0 .. n/2
  const int nout = ax == 0 ? e0 : (ax == 1 ? e1 : e2);
  const int nh = n / 2 + 1;
  for (int i = threadIdx.x; i < nout * nh; i += blockDim.x) {
    const int f = i / nout, a = i - f * nout;
    Ms[i] = M[(int64_t)a * n + f];
  }
  __syncthreads();
  const int ea = ax == 0 ? e1 : e0, eb = ax == 2 ? e1 : e2;
  const int64_t sa_in = ax == 0 ? vin.s1 : vin.s0, sb_in = ax == 2 ? vin.s1 : vin.s2;
  const int64_t sa_out = ax == 0 ? vout.s1 : vout.s0, sb_out = ax == 2 ? vout.s1 : vout.s2;
  const int64_t step_in = ax == 0 ? vin.s0 : (ax == 1 ? vin.s1 : vin.s2);
  const int64_t step_out = ax == 0 ? vout.s0 : (ax == 1 ? vout.s1 : vout.s2);
  const int CL = C / LPT;
  const int64_t lines = B * ea * eb * (int64_t)CL;
  const int np = (n - 1) / 2;     // conjugate pairs (f, n - f), f = 1 .. np
  const bool mid = (n % 2) == 0;  // f = n/2 pairs with itself
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < lines;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t t = idx;
    const int c = (int)(t % CL) * LPT;
    t /= CL;
    const int ib = (int)(t % eb);
    t /= eb;
    const int ia = (int)(t % ea);
    const int64_t b = t / ea;
    const T* ip = in + b * vin.sb + ia * sa_in + ib * sb_in + c;
    T acc[AMAX][LPT];
    {
      T v0[LPT];
#pragma unroll
      for (int l = 0; l < LPT; ++l) v0[l] = ip[l];
#pragma unroll
      for (int a = 0; a < AMAX; ++a)
        if (a < nout) {
          const T m = Ms[a];
#pragma unroll
          for (int l = 0; l < LPT; ++l) acc[a][l] = cmul(m, v0[l]);
        }
    }
    T z1[LPT], z2[LPT];
#pragma unroll
    for (int l = 0; l < LPT; ++l) {
      z1[l] = np > 0 ? ip[step_in + l] : mk<R>(0, 0);
      z2[l] = np > 0 ? ip[(int64_t)(n - 1) * step_in + l] : mk<R>(0, 0);
    }
    for (int f = 1; f <= np; ++f) {
      T u[LPT], w[LPT];
#pragma unroll
      for (int l = 0; l < LPT; ++l) {
        u[l] = mk<R>(z1[l].x + z2[l].x, z1[l].y + z2[l].y);
        w[l] = mk<R>(z1[l].x - z2[l].x, z1[l].y - z2[l].y);
      }
      if (f < np) {  // next pair's loads in flight during this pair's products
#pragma unroll
        for (int l = 0; l < LPT; ++l) {
          z1[l] = ip[(int64_t)(f + 1) * step_in + l];
          z2[l] = ip[(int64_t)(n - f - 1) * step_in + l];
        }
      }
      const T* Mr = Ms + f * nout;
#pragma unroll
      for (int a = 0; a < AMAX; ++a)
        if (a < nout) {
          const T m = Mr[a];
#pragma unroll
          for (int l = 0; l < LPT; ++l) {
            acc[a][l].x = fma(m.x, u[l].x, acc[a][l].x);
            acc[a][l].x = fma(-m.y, w[l].y, acc[a][l].x);
            acc[a][l].y = fma(m.x, u[l].y, acc[a][l].y);
            acc[a][l].y = fma(m.y, w[l].x, acc[a][l].y);
          }
        }
    }
    if (mid) {
      const T* Mr = Ms + (n / 2) * nout;
      T vm[LPT];
#pragma unroll
      for (int l = 0; l < LPT; ++l) vm[l] = ip[(int64_t)(n / 2) * step_in + l];
#pragma unroll
      for (int a = 0; a < AMAX; ++a)
        if (a < nout)
#pragma unroll
          for (int l = 0; l < LPT; ++l) cfma(acc[a][l], Mr[a], vm[l]);
    }
    T* op = out + b * vout.sb + ia * sa_out + ib * sb_out + c;
#pragma unroll
    for (int a = 0; a < AMAX; ++a)
      if (a < nout)
#pragma unroll
        for (int l = 0; l < LPT; ++l) op[a * step_out + l] = acc[a][l];
  }
}

// Fused second and third passes (FP32, 32 channels), one block per
// (box, x-frequency) slab.  Forward: the slab t[b][fx][y][z][c] (SP x SP x 32
// values, the output of the x pass) is staged in shared memory; a warp takes
// a pair of y-frequencies (fy, n - fy), lane = channel, forms the two rows
// T[z] of the y pass in registers (the conjugate-row pairing of the line
// kernels) and from each row the n z-frequencies, which it stores straight
// into the spectrum layout Q[fx][fy][fz][b][c] (256 contiguous bytes per
// warp store).  The y-pass intermediate never goes to HBM: per box the pass
// pair reads n SP^2 and writes n^3 values instead of reading and writing
// n SP^2 + n^2 SP.
template <int SP>
__global__ void __launch_bounds__(256, 2) k_dft_fwd_yz(const float2* __restrict__ in, float2* __restrict__ out,
                                                    int64_t B, const float2* __restrict__ M, int n) {
  extern __shared__ float4 fyz_smem[];
  float2* slab = reinterpret_cast<float2*>(fyz_smem);  // [SP][SP][32]
  float2* Ms = slab + SP * SP * 32;                    // rows 0 .. n/2 of M, [f][SP]
  const int nh = n / 2 + 1;
  const int64_t sl = blockIdx.x;
  const int64_t b = sl / n;
  const int fx = (int)(sl - b * n);
  {
    const float4* src = reinterpret_cast<const float4*>(in + sl * (SP * SP * 32));
    float4* dst = reinterpret_cast<float4*>(slab);
    for (int i = threadIdx.x; i < SP * SP * 16; i += blockDim.x) dst[i] = src[i];
    for (int i = threadIdx.x; i < nh * SP; i += blockDim.x) Ms[i] = M[i];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int64_t fstride = B * 32;  // between consecutive z-frequencies
  for (int fy = warp; fy < nh; fy += nw) {
    // y pass: a[z] = (S1, S3), c[z] = (S2, S4) over the slab's y lines
    float2 t0[SP], t1[SP];
#pragma unroll
    for (int z = 0; z < SP; ++z) t0[z] = t1[z] = make_float2(0.f, 0.f);
    const float2* Mr = Ms + fy * SP;
#pragma unroll 1
    for (int y = 0; y < SP; ++y) {
      const float2 m = Mr[y];
      const float2* sv = slab + y * SP * 32 + lane;
#pragma unroll
      for (int z = 0; z < SP; ++z) {
        const float2 v = sv[z * 32];
        t0[z].x = fmaf(m.x, v.x, t0[z].x);
        t0[z].y = fmaf(m.x, v.y, t0[z].y);
        t1[z].x = fmaf(m.y, v.y, t1[z].x);
        t1[z].y = fmaf(m.y, v.x, t1[z].y);
      }
    }
    // rows fy and n - fy: (S1 - S2) + i (S3 + S4) and (S1 + S2) + i (S3 - S4)
#pragma unroll
    for (int z = 0; z < SP; ++z) {
      const float2 a = t0[z], c = t1[z];
      t0[z] = make_float2(a.x - c.x, a.y + c.y);
      t1[z] = make_float2(a.x + c.x, a.y - c.y);
    }
    const bool ypair = fy != 0 && 2 * fy != n;
    for (int r = 0; r < (ypair ? 2 : 1); ++r) {
      const int fyr = r == 0 ? fy : n - fy;
      float2* op = out + (((int64_t)fx * n + fyr) * n * B + b) * 32 + lane;
      for (int fz = 0; fz < nh; ++fz) {
        const float2* Mz = Ms + fz * SP;
        float s1 = 0.f, s2 = 0.f, s3 = 0.f, s4 = 0.f;
#pragma unroll
        for (int z = 0; z < SP; ++z) {
          const float2 m = Mz[z];
          const float2 v = r == 0 ? t0[z] : t1[z];
          s1 = fmaf(m.x, v.x, s1);
          s2 = fmaf(m.y, v.y, s2);
          s3 = fmaf(m.x, v.y, s3);
          s4 = fmaf(m.y, v.x, s4);
        }
        op[fz * fstride] = make_float2(s1 - s2, s3 + s4);
        if (fz != 0 && 2 * fz != n) op[(int64_t)(n - fz) * fstride] = make_float2(s1 + s2, s3 - s4);
      }
    }
  }
}

// Inverse counterpart: the z and y inverse passes of one (box, x-frequency)
// slab.  Phase 1: a warp takes a y-frequency row, lane = channel, reads its n
// spectrum values (256 bytes per warp load) and forms the SP outputs of the
// z pass (conjugate input pairs folded as in k_dft_inv_line) into shared
// memory U[fy][z][c].  Phase 2: a warp takes output points (y, z) and folds
// the y-frequency pairs of U into t[b][fx][y][z][c], the input of the x pass.
template <int SP>
__global__ void __launch_bounds__(256) k_dft_inv_zy(const float2* __restrict__ in, float2* __restrict__ out,
                                                    int64_t B, const float2* __restrict__ M, int n) {
  extern __shared__ float4 izy_smem[];
  float2* U = reinterpret_cast<float2*>(izy_smem);  // [n][SP][32]
  float2* Ms = U + (int64_t)n * SP * 32;            // [f][a] = M[a][f], f = 0 .. n/2
  const int nh = n / 2 + 1;
  const int np = (n - 1) / 2;
  const bool mid = (n % 2) == 0;
  for (int i = threadIdx.x; i < nh * SP; i += blockDim.x) {
    const int f = i / SP, a = i - f * SP;
    Ms[i] = M[(int64_t)a * n + f];
  }
  __syncthreads();
  const int64_t sl = blockIdx.x;
  const int64_t b = sl / n;
  const int fx = (int)(sl - b * n);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int64_t fstride = B * 32;
  for (int fy = warp; fy < n; fy += nw) {
    const float2* ip = in + (((int64_t)fx * n + fy) * n * B + b) * 32 + lane;
    float2 acc[SP];
    {
      const float2 v0 = ip[0];
#pragma unroll
      for (int a = 0; a < SP; ++a) {
        const float2 m = Ms[a];
        acc[a] = make_float2(m.x * v0.x - m.y * v0.y, m.x * v0.y + m.y * v0.x);
      }
    }
    for (int f = 1; f <= np; ++f) {
      const float2 z1 = ip[f * fstride], z2 = ip[(int64_t)(n - f) * fstride];
      const float2 u = make_float2(z1.x + z2.x, z1.y + z2.y), w = make_float2(z1.x - z2.x, z1.y - z2.y);
      const float2* Mr = Ms + f * SP;
#pragma unroll
      for (int a = 0; a < SP; ++a) {
        const float2 m = Mr[a];
        acc[a].x = fmaf(m.x, u.x, acc[a].x);
        acc[a].x = fmaf(-m.y, w.y, acc[a].x);
        acc[a].y = fmaf(m.x, u.y, acc[a].y);
        acc[a].y = fmaf(m.y, w.x, acc[a].y);
      }
    }
    if (mid) {
      const float2 vm = ip[(int64_t)(n / 2) * fstride];
      const float2* Mr = Ms + (n / 2) * SP;
#pragma unroll
      for (int a = 0; a < SP; ++a) {
        const float2 m = Mr[a];
        acc[a].x = fmaf(m.x, vm.x, fmaf(-m.y, vm.y, acc[a].x));
        acc[a].y = fmaf(m.x, vm.y, fmaf(m.y, vm.x, acc[a].y));
      }
    }
#pragma unroll
    for (int a = 0; a < SP; ++a) U[(fy * SP + a) * 32 + lane] = acc[a];
  }
  __syncthreads();
  float2* op = out + sl * (SP * SP * 32) + lane;
  for (int o = warp; o < SP * SP; o += nw) {
    const int y = o / SP, z = o - y * SP;
    const float2 m0 = Ms[y], v0 = U[z * 32 + lane];
    float ax = m0.x * v0.x - m0.y * v0.y, ay = m0.x * v0.y + m0.y * v0.x;
    for (int f = 1; f <= np; ++f) {
      const float2 z1 = U[(f * SP + z) * 32 + lane], z2 = U[((n - f) * SP + z) * 32 + lane];
      const float2 m = Ms[f * SP + y];
      ax = fmaf(m.x, z1.x + z2.x, ax);
      ax = fmaf(-m.y, z1.y - z2.y, ax);
      ay = fmaf(m.x, z1.y + z2.y, ay);
      ay = fmaf(m.y, z1.x - z2.x, ay);
    }
    if (mid) {
      const float2 m = Ms[(n / 2) * SP + y], vm = U[((n / 2) * SP + z) * 32 + lane];
      ax = fmaf(m.x, vm.x, fmaf(-m.y, vm.y, ax));
      ay = fmaf(m.x, vm.y, fmaf(m.y, vm.x, ay));
    }
    op[(int64_t)o * 32] = make_float2(ax, ay);
  }
}

// Whether the fused forward (y, z) / inverse (z, y) passes take a level of
// sp splines per axis and FFT length n (9, 13 or 21 splines; shared memory).
static size_t dft_yz_smem(int sp, int n, bool inverse) {
  const int nh = n / 2 + 1;
  return inverse ? sizeof(float2) * ((size_t)n * sp * 32 + (size_t)nh * sp)
                 : sizeof(float2) * ((size_t)sp * sp * 32 + (size_t)nh * sp);
}
bool dft_yz_fits(int sp, int n) { return (sp == 9 || sp == 13 || sp == 21) && dft_yz_smem(sp, n, false) <= 200 * 1024; }
bool dft_zy_fits(int sp, int n) { return (sp == 9 || sp == 13 || sp == 21) && dft_yz_smem(sp, n, true) <= 200 * 1024; }

// Fused y-z forward (in: t[b][fx][y][z][32] -> out: Q[fx][fy][fz][b][32]) or
// z-y inverse (in: Q layout -> out: t layout).  Returns false when they do not
// apply (splines per axis other than 9, 13 or 21, or shared memory).
bool launch_dft_yz(const float2* in, float2* out, int64_t B, int sp, int n, const float2* M, bool inverse,
                   cudaStream_t s) {
  const int64_t slabs = B * (int64_t)n;
  if (slabs <= 0) return true;
  if (slabs > 0x7FFFFFFFLL) return false;
  const size_t smem = dft_yz_smem(sp, n, inverse);
  if (smem > 200 * 1024) return false;
#define EFIE_YZ(SPV)                                                                                 \
  if (sp == SPV) {                                                                                   \
    if (inverse) {                                                                                   \
      static SmemAttr attr;                                                                          \
      smem_attr_once(k_dft_inv_zy<SPV>, (int)smem, attr.v);                                          \
      k_dft_inv_zy<SPV><<<(unsigned)slabs, 256, smem, s>>>(in, out, B, M, n);                        \
    } else {                                                                                         \
      static SmemAttr attr;                                                                          \
      smem_attr_once(k_dft_fwd_yz<SPV>, (int)smem, attr.v);                                          \
      k_dft_fwd_yz<SPV><<<(unsigned)slabs, 256, smem, s>>>(in, out, B, M, n);                        \
    }                                                                                                \
    return true;                                                                                     \
  }
  EFIE_YZ(9)
  EFIE_YZ(13)
  EFIE_YZ(21)
#undef EFIE_YZ
  return false;
}

// forward (inverse = false: M is n x nin, nin inputs -> n outputs along ax) or
// inverse (M is nout x n, n inputs -> nout outputs); returns false when no
// specialisation fits (the caller then uses launch_mode)
template <typename R>
bool launch_dft(const cpx_t<R>* in, View vin, cpx_t<R>* out, View vout, int64_t B, int C, int ax, int nin,
                int e0, int e1, int e2, const cpx_t<R>* M, int n, bool inverse, cudaStream_t s) {
  using T = cpx_t<R>;
  const int ea = ax == 0 ? e1 : e0, eb = ax == 2 ? e1 : e2;
  const int nout = ax == 0 ? e0 : (ax == 1 ? e1 : e2);
  const int nh = n / 2 + 1;
  const bool two = (C % 2) == 0 && sizeof(R) == 4;
  const int lpt = two ? 2 : 1;
  const int64_t lines = B * ea * eb * (int64_t)(C / lpt);
  if (lines <= 0) return true;
  int64_t blocks = ceil_div(lines, 128);
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (!inverse) {
    const size_t smem = sizeof(T) * (size_t)nh * nin;
    if (smem > 96 * 1024) return false;
#define EFIE_DF(NM)                                                                                          \
  if (nin <= NM) {                                                                                           \
    if (two && NM <= 21) {                                                                                   \
      auto k = k_dft_fwd_line<R, NM, (sizeof(R) == 4 && NM <= 21) ? 2 : 1>;                                  \
      static SmemAttr attr;                                                                  \
      smem_attr_once(k, 96 * 1024, attr.v);                                                                    \
      k<<<(unsigned)blocks, 128, smem, s>>>(in, vin, out, vout, B, C, ax, nin, e0, e1, e2, M, n);            \
      return true;                                                                                           \
    }                                                                                                        \
    const int64_t lines1 = B * ea * eb * (int64_t)C;                                                         \
    int64_t blocks1 = ceil_div(lines1, 128);                                                                 \
    if (blocks1 > 152 * 32) blocks1 = 152 * 32;                                                              \
    auto k = k_dft_fwd_line<R, NM, 1>;                                                                       \
    static SmemAttr attr1;                                                                   \
    smem_attr_once(k, 96 * 1024, attr1.v);                                                                     \
    k<<<(unsigned)blocks1, 128, smem, s>>>(in, vin, out, vout, B, C, ax, nin, e0, e1, e2, M, n);             \
    return true;                                                                                             \
  }
    EFIE_DF(9)
    EFIE_DF(13)
    EFIE_DF(21)
    EFIE_DF(40)
#undef EFIE_DF
    return false;
  }
  const size_t smem = sizeof(T) * (size_t)nout * nh;
  if (smem > 96 * 1024) return false;
#define EFIE_DI(AM)                                                                                          \
  if (nout <= AM) {                                                                                          \
    if (two && AM <= 21) {                                                                                   \
      auto k = k_dft_inv_line<R, AM, (sizeof(R) == 4 && AM <= 21) ? 2 : 1>;                                  \
      static SmemAttr attr;                                                                  \
      smem_attr_once(k, 96 * 1024, attr.v);                                                                    \
      k<<<(unsigned)blocks, 128, smem, s>>>(in, vin, out, vout, B, C, ax, nin, e0, e1, e2, M, n);            \
      return true;                                                                                           \
    }                                                                                                        \
    const int64_t lines1 = B * ea * eb * (int64_t)C;                                                         \
    int64_t blocks1 = ceil_div(lines1, 128);                                                                 \
    if (blocks1 > 152 * 32) blocks1 = 152 * 32;                                                              \
    auto k = k_dft_inv_line<R, AM, 1>;                                                                       \
    static SmemAttr attr1;                                                                   \
    smem_attr_once(k, 96 * 1024, attr1.v);                                                                     \
    k<<<(unsigned)blocks1, 128, smem, s>>>(in, vin, out, vout, B, C, ax, nin, e0, e1, e2, M, n);             \
    return true;                                                                                             \
  }
  EFIE_DI(9)
  EFIE_DI(13)
  EFIE_DI(21)
#undef EFIE_DI
  return false;
}

template <typename R>
void launch_mode(const cpx_t<R>* in, View vin, cpx_t<R>* out, View vout, int64_t B, int C, int ax,
                 int nin, int e0, int e1, int e2, const void* M0, const void* M1, bool complex_m,
                 const int8_t* sel, const int64_t* srcmap, bool accumulate, cudaStream_t s) {
  int64_t total = B * e0 * e1 * e2 * (int64_t)C;
  if (total <= 0) return;
  const int nout = ax == 0 ? e0 : (ax == 1 ? e1 : e2);
  const size_t esz = complex_m ? sizeof(cpx_t<R>) : sizeof(R);
  const size_t smem = (size_t)nout * nin * esz * ((M1 && M1 != M0) ? 2 : 1);
  if (smem <= 96 * 1024) {
    bool done = complex_m ? dispatch_mode_line<R, true>(in, vin, out, vout, B, C, ax, nin, e0, e1, e2, M0, M1, sel,
                                                        srcmap, accumulate, smem, s)
                          : dispatch_mode_line<R, false>(in, vin, out, vout, B, C, ax, nin, e0, e1, e2, M0, M1,
                                                         sel, srcmap, accumulate, smem, s);
    if (done) return;
  }
  int64_t blocks = ceil_div(total, 256);
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (complex_m)
    k_mode<R, true><<<(unsigned)blocks, 256, 0, s>>>(in, vin, out, vout, B, C, ax, nin, e0, e1, e2, M0,
                                                     M1, sel, srcmap, accumulate);
  else
    k_mode<R, false><<<(unsigned)blocks, 256, 0, s>>>(in, vin, out, vout, B, C, ax, nin, e0, e1, e2, M0,
                                                      M1, sel, srcmap, accumulate);
}

// ---------------------------------------------------------------- leaf grids
// Channel order inside a grid point: c = d * nr + r (component d = 0..2 the
// vector part, 3 the charge part; r the right-hand side), so the vector part
// of one point is 3 nr contiguous values and the charge part nr more.

// Gather lists (setup): the moments re-indexed by grid point.  For leaf box b
// and point pt of its sp^3 grid, entries [ptr[pt], ptr[pt+1]) (offsets within
// the box) hold (k, m_0, m_1, m_2) for every RWG k of the box (local index)
// whose moment block covers pt, in increasing k; triangles likewise hold
// (t, m^phi).  A box's entries start where its RWGs' moment data starts
// (mr_off / 3, mt_off), since both orderings hold the same entries.  One CTA
// per box, one thread per point; the covering test reads each basis
// function's base and extents, so the lists are deterministic.
// Points are taken GB_PTS at a time (the per-point counters live in shared
// memory), so leaves of any spline count fit; thread 0 carries the running
// list offsets from one group of points to the next.
constexpr int GB_PTS = 8192;

template <typename R>
__global__ void k_gather_build(const R* __restrict__ mr, const int32_t* __restrict__ mr_base,
                               const int32_t* __restrict__ mr_ext, const int64_t* __restrict__ mr_off,
                               const R* __restrict__ mt, const int32_t* __restrict__ mt_base,
                               const int32_t* __restrict__ mt_ext, const int64_t* __restrict__ mt_off,
                               const int64_t* __restrict__ box_rwg_ptr, const int64_t* __restrict__ box_tri_ptr,
                               int sp, int32_t* __restrict__ gptr_r, int32_t* __restrict__ gptr_t,
                               R* __restrict__ gr, R* __restrict__ gt) {
  extern __shared__ int32_t gcnt[];  // [2][min(npts, GB_PTS)]
  const int b = blockIdx.x, npts = sp * sp * sp;
  const int gp = npts < GB_PTS ? npts : GB_PTS;
  const int64_t k0 = box_rwg_ptr[b], k1 = box_rwg_ptr[b + 1];
  const int64_t t0 = box_tri_ptr[b], t1 = box_tri_ptr[b + 1];
  auto covers = [&](const int32_t* base, const int32_t* ext, int64_t i, int p0, int p1, int p2, int& e) {
    const int a0 = p0 - base[3 * i], a1 = p1 - base[3 * i + 1], a2 = p2 - base[3 * i + 2];
    const int e0 = ext[3 * i], e1 = ext[3 * i + 1], e2 = ext[3 * i + 2];
    if ((unsigned)a0 >= (unsigned)e0 || (unsigned)a1 >= (unsigned)e1 || (unsigned)a2 >= (unsigned)e2) return false;
    e = (a0 * e1 + a1) * e2 + a2;
    return true;
  };
  int32_t* pr = gptr_r + (int64_t)b * (npts + 1);
  int32_t* pt_ = gptr_t + (int64_t)b * (npts + 1);
  R* outr = gr + 4 * (k0 < k1 ? mr_off[k0] / 3 : 0);
  R* outt = gt + 2 * (t0 < t1 ? mt_off[t0] : 0);
  int32_t rr = 0, rt = 0;  // running offsets (thread 0)
  for (int q0 = 0; q0 < npts; q0 += gp) {
    const int q1 = q0 + gp < npts ? q0 + gp : npts;
    for (int pt = q0 + threadIdx.x; pt < q1; pt += blockDim.x) {
      const int p0 = pt / (sp * sp), p1 = (pt / sp) % sp, p2 = pt % sp;
      int cr = 0, ct = 0, e;
      for (int64_t i = k0; i < k1; ++i) cr += covers(mr_base, mr_ext, i, p0, p1, p2, e);
      for (int64_t i = t0; i < t1; ++i) ct += covers(mt_base, mt_ext, i, p0, p1, p2, e);
      gcnt[pt - q0] = cr;
      gcnt[gp + pt - q0] = ct;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int pt = q0; pt < q1; ++pt) {
        const int32_t vr = gcnt[pt - q0], vt = gcnt[gp + pt - q0];
        gcnt[pt - q0] = rr;
        gcnt[gp + pt - q0] = rt;
        pr[pt] = rr;
        pt_[pt] = rt;
        rr += vr;
        rt += vt;
      }
      if (q1 == npts) {
        pr[npts] = rr;
        pt_[npts] = rt;
      }
    }
    __syncthreads();
    for (int pt = q0 + threadIdx.x; pt < q1; pt += blockDim.x) {
      const int p0 = pt / (sp * sp), p1 = (pt / sp) % sp, p2 = pt % sp;
      int64_t pos = gcnt[pt - q0];
      int e;
      for (int64_t i = k0; i < k1; ++i)
        if (covers(mr_base, mr_ext, i, p0, p1, p2, e)) {
          const R* m = mr + mr_off[i] + 3 * e;
          R* o = outr + 4 * pos++;
          o[0] = (R)(i - k0);
          o[1] = m[0];
          o[2] = m[1];
          o[3] = m[2];
        }
      pos = gcnt[gp + pt - q0];
      for (int64_t i = t0; i < t1; ++i)
        if (covers(mt_base, mt_ext, i, p0, p1, p2, e)) {
          R* o = outt + 2 * pos++;
          o[0] = (R)(i - t0);
          o[1] = mt[mt_off[i] + e];
        }
    }
    __syncthreads();  // gcnt is reused by the next group of points
  }
}

// ---------------------------------------------------------------- anterpolation
// q[b][pt][d nr + r] = sum over the gather list of pt: m_d x_r[k] (d < 3) and
// sum of m^phi rho_r[t] (d = 3).  One CTA per leaf box; the box's currents and
// charges are staged in shared memory (AK basis functions at a time; boxes
// with more take several passes over their sorted lists).  A warp takes four
// grid points at a time, lane = (point, right-hand side): the eight lanes of a
// point read the same list entry (one broadcast) and eight consecutive staged
// values, and own their 4 output components outright -- no atomics, no
// reductions, each moment entry read once per launch, each output written once.
template <typename R>
struct AnterpCfg;
template <>
struct AnterpCfg<float> {
  static constexpr int AK = 256, XS = 10;  // 80-byte rows
};
template <>
struct AnterpCfg<double> {
  static constexpr int AK = 128, XS = 9;   // 144-byte rows
};

template <typename R>
__global__ void __launch_bounds__(256) k_anterp(const R* __restrict__ gr, const R* __restrict__ gt,
                                                const int32_t* __restrict__ gptr_r,
                                                const int32_t* __restrict__ gptr_t,
                                                const int64_t* __restrict__ mr_off,
                                                const int64_t* __restrict__ mt_off,
                                                const int64_t* __restrict__ box_rwg_ptr,
                                                const int64_t* __restrict__ box_tri_ptr,
                                                const int32_t* __restrict__ out_box,
                                                const cpx_t<R>* __restrict__ xs, int64_t ldx,
                                                const cpx_t<R>* __restrict__ rho, int64_t ldr, int nr,
                                                cpx_t<R>* __restrict__ q, int sp) {
  using T = cpx_t<R>;
  constexpr int AK = AnterpCfg<R>::AK, XS = AnterpCfg<R>::XS;
  __shared__ __align__(16) T xsm[AK][XS];
  __shared__ __align__(16) T rsm[AK][XS];
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int npts = sp * sp * sp;
  const int64_t k0 = box_rwg_ptr[b], t0 = box_tri_ptr[b];
  const int nk = (int)(box_rwg_ptr[b + 1] - k0), nt = (int)(box_tri_ptr[b + 1] - t0);
  const R* ger = gr + 4 * (nk > 0 ? mr_off[k0] / 3 : 0);
  const R* get = gt + 2 * (nt > 0 ? mt_off[t0] : 0);
  const int32_t* pr = gptr_r + (int64_t)b * (npts + 1);
  const int32_t* pq = gptr_t + (int64_t)b * (npts + 1);
  const int nchunk = max((nk + AK - 1) / AK, (nt + AK - 1) / AK);
  auto stage = [&](int c) {
    for (int i = tid; i < AK * nr; i += blockDim.x) {
      const int r = i / AK, kk = i - r * AK, k = c * AK + kk;
      if (k < nk) xsm[kk][r] = xs[r * ldx + k0 + k];
      if (k < nt) rsm[kk][r] = rho[r * ldr + t0 + k];
    }
  };
  if (nchunk == 1) {
    stage(0);
    __syncthreads();
  }
  const int r = lane & 7, ps = lane >> 3;
  const int C = 4 * nr;
  const int per_pass = 4 * (blockDim.x >> 5);
  for (int pb = 0; pb < npts; pb += per_pass) {
    const int p = pb + 4 * warp + ps;
    const bool okp = p < npts;
    T a0 = mk<R>(0, 0), a1 = a0, a2 = a0, a3 = a0;
    int er = okp ? pr[p] : 0, er1 = okp ? pr[p + 1] : 0;
    int et = okp ? pq[p] : 0, et1 = okp ? pq[p + 1] : 0;
    for (int c = 0; c < nchunk; ++c) {
      if (nchunk > 1) {
        __syncthreads();
        stage(c);
        __syncthreads();
      }
      const R kc0 = (R)(c * AK), kc1 = (R)((c + 1) * AK);
      auto load4 = [&](int64_t i, R& ek, R& m0, R& m1, R& m2) {
        const R* e = ger + 4 * i;
        if constexpr (sizeof(R) == 4) {
          const float4 v = *reinterpret_cast<const float4*>(e);
          ek = v.x, m0 = v.y, m1 = v.z, m2 = v.w;
        } else {
          const double2 v0 = *reinterpret_cast<const double2*>(e), v1 = *reinterpret_cast<const double2*>(e + 2);
          ek = v0.x, m0 = v0.y, m1 = v1.x, m2 = v1.y;
        }
      };
      auto mac3 = [&](R ek, R m0, R m1, R m2) {
        const T xv = xsm[(int)(ek - kc0)][r];
        a0.x = fma(m0, xv.x, a0.x);
        a0.y = fma(m0, xv.y, a0.y);
        a1.x = fma(m1, xv.x, a1.x);
        a1.y = fma(m1, xv.y, a1.y);
        a2.x = fma(m2, xv.x, a2.x);
        a2.y = fma(m2, xv.y, a2.y);
      };
      if (nchunk == 1) {
        // every entry belongs to this chunk: four list entries in flight at a time
        for (; er + 3 < er1; er += 4) {
          R k_[4], x_[4], y_[4], z_[4];
#pragma unroll
          for (int t = 0; t < 4; ++t) load4(er + t, k_[t], x_[t], y_[t], z_[t]);
#pragma unroll
          for (int t = 0; t < 4; ++t) mac3(k_[t], x_[t], y_[t], z_[t]);
        }
      }
      for (; er < er1; ++er) {
        R ek, m0, m1, m2;
        load4(er, ek, m0, m1, m2);
        if (ek >= kc1) break;
        mac3(ek, m0, m1, m2);
      }
      auto load2 = [&](int64_t i, R& ek, R& m) {
        const R* e = get + 2 * i;
        if constexpr (sizeof(R) == 4) {
          const float2 v = *reinterpret_cast<const float2*>(e);
          ek = v.x, m = v.y;
        } else {
          const double2 v = *reinterpret_cast<const double2*>(e);
          ek = v.x, m = v.y;
        }
      };
      auto mac1 = [&](R ek, R m) {
        const T v = rsm[(int)(ek - kc0)][r];
        a3.x = fma(m, v.x, a3.x);
        a3.y = fma(m, v.y, a3.y);
      };
      if (nchunk == 1) {
        for (; et + 3 < et1; et += 4) {
          R k_[4], m_[4];
#pragma unroll
          for (int t = 0; t < 4; ++t) load2(et + t, k_[t], m_[t]);
#pragma unroll
          for (int t = 0; t < 4; ++t) mac1(k_[t], m_[t]);
        }
      }
      for (; et < et1; ++et) {
        R ek, m;
        load2(et, ek, m);
        if (ek >= kc1) break;
        mac1(ek, m);
      }
    }
    if (okp && r < nr) {
      T* qp = q + ((int64_t)(out_box ? out_box[b] : b) * npts + p) * C + r;
      qp[0] = a0;
      qp[nr] = a1;
      qp[2 * nr] = a2;
      qp[3 * nr] = a3;
    }
  }
}

template <typename R>
void launch_gather_build(const R* mr, const int32_t* mr_base, const int32_t* mr_ext, const int64_t* mr_off,
                         const R* mt, const int32_t* mt_base, const int32_t* mt_ext, const int64_t* mt_off,
                         const int64_t* box_rwg_ptr, const int64_t* box_tri_ptr, int64_t B, int sp,
                         int32_t* gptr_r, int32_t* gptr_t, R* gr, R* gt, cudaStream_t s) {
  if (B <= 0) return;
  const int64_t npts = (int64_t)sp * sp * sp;
  const size_t smem = sizeof(int32_t) * 2 * (size_t)(npts < GB_PTS ? npts : GB_PTS);
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_gather_build<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_gather_build<R><<<(unsigned)B, 256, smem, s>>>(mr, mr_base, mr_ext, mr_off, mt, mt_base, mt_ext, mt_off,
                                                   box_rwg_ptr, box_tri_ptr, sp, gptr_r, gptr_t, gr, gt);
}

template <typename R>
void launch_anterp(const R* gr, const R* gt, const int32_t* gptr_r, const int32_t* gptr_t, const int64_t* mr_off,
                   const int64_t* mt_off, const int64_t* box_rwg_ptr, const int64_t* box_tri_ptr, int64_t B,
                   const int32_t* out_box, const cpx_t<R>* xs, int64_t ldx, const cpx_t<R>* rho, int64_t ldr, int nr,
                   cpx_t<R>* q, int sp, cudaStream_t s) {
  if (B <= 0 || nr <= 0) return;
  k_anterp<R><<<(unsigned)B, 256, 0, s>>>(gr, gt, gptr_r, gptr_t, mr_off, mt_off, box_rwg_ptr, box_tri_ptr, out_box,
                                          xs, ldx, rho, ldr, nr, q, sp);
}

// ---------------------------------------------------------------- interpolation
// yA[r][i] = sum_e sum_d m_d[e] r[b][pt(e)][d nr + r] for RWG i, and
// u[r][t] = sum_e m^phi[e] r[b][pt(e)][3 nr + r] for triangle t (FP64
// outputs).  One warp per basis function.  RWG: lane = channel d nr + r of
// the vector part (3 nr <= 24 lanes), so every grid point is one coalesced
// read; the three components are summed by shuffles at the end.  Triangle:
// the charge part is nr values per point, so the warp takes 32/nr entries at
// a time, lane = (entry slot, r).
template <typename R>
__global__ void __launch_bounds__(256) k_interp(const R* __restrict__ mr, const int32_t* __restrict__ mr_base,
                                                const int32_t* __restrict__ mr_ext,
                                                const int64_t* __restrict__ mr_off,
                                                const int32_t* __restrict__ rwg_box, int64_t N,
                                                const R* __restrict__ mt, const int32_t* __restrict__ mt_base,
                                                const int32_t* __restrict__ mt_ext,
                                                const int64_t* __restrict__ mt_off,
                                                const int32_t* __restrict__ tri_box, int64_t Nt,
                                                const cpx_t<R>* __restrict__ rg, int sp, int nr,
                                                double2* __restrict__ yA, int64_t ldy, double2* __restrict__ u,
                                                int64_t ldu) {
  using T = cpx_t<R>;
  const int lane = threadIdx.x & 31;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= N + Nt) return;
  const int npts = sp * sp * sp, C = 4 * nr;
  T acc = mk<R>(0, 0);
  if (w < N) {
    const int64_t i = w;
    const int b0 = mr_base[3 * i], b1 = mr_base[3 * i + 1], b2 = mr_base[3 * i + 2];
    const int e0 = mr_ext[3 * i], e1 = mr_ext[3 * i + 1], e2 = mr_ext[3 * i + 2];
    const int ne = e0 * e1 * e2;
    const bool act = lane < 3 * nr;
    const int d = act ? lane / nr : 0;
    const R* m = mr + mr_off[i] + d;  // entry e at m[3 e]
    const T* gp = rg + (int64_t)rwg_box[i] * npts * C + lane;
    if (act && ne > 0) {
      int e = 0;
      for (int a0 = 0; a0 < e0; ++a0)
        for (int a1 = 0; a1 < e1; ++a1) {
          const T* gl = gp + (int64_t)(((b0 + a0) * sp + b1 + a1) * sp + b2) * C;
          const R* ml = m + 3 * e;
#pragma unroll 4
          for (int a2 = 0; a2 < e2; ++a2) {
            const R mv = ml[3 * a2];
            const T gv = gl[a2 * C];
            acc.x = fma(mv, gv.x, acc.x);
            acc.y = fma(mv, gv.y, acc.y);
          }
          e += e2;
        }
    }
    R sx = acc.x + __shfl_down_sync(0xffffffffu, acc.x, nr) + __shfl_down_sync(0xffffffffu, acc.x, 2 * nr);
    R sy = acc.y + __shfl_down_sync(0xffffffffu, acc.y, nr) + __shfl_down_sync(0xffffffffu, acc.y, 2 * nr);
    if (lane < nr) yA[lane * ldy + i] = make_double2((double)sx, (double)sy);
  } else {
    const int64_t i = w - N;
    const int b0 = mt_base[3 * i], b1 = mt_base[3 * i + 1], b2 = mt_base[3 * i + 2];
    const int e0 = mt_ext[3 * i], e1 = mt_ext[3 * i + 1], e2 = mt_ext[3 * i + 2];
    const int ne = e0 * e1 * e2;
    const int Q = 32 / nr;
    const int slot = lane / nr, r = lane - slot * nr;
    const R* m = mt + mt_off[i];
    const T* gp = rg + (int64_t)tri_box[i] * npts * C + 3 * nr + r;
    if (slot < Q && ne > 0) {
      int e = slot;
      int a0 = e / (e1 * e2), a1 = (e / e2) % e1, a2 = e % e2;
      for (; e < ne; e += Q) {
        const T gv = gp[(int64_t)(((b0 + a0) * sp + b1 + a1) * sp + b2 + a2) * C];
        const R mv = m[e];
        acc.x = fma(mv, gv.x, acc.x);
        acc.y = fma(mv, gv.y, acc.y);
        a2 += Q;
        while (a2 >= e2) {
          a2 -= e2;
          if (++a1 == e1) {
            a1 = 0;
            ++a0;
          }
        }
      }
    }
    R sx = acc.x, sy = acc.y;
    for (int o = 1; o < Q; ++o) {
      sx += __shfl_down_sync(0xffffffffu, acc.x, o * nr);
      sy += __shfl_down_sync(0xffffffffu, acc.y, o * nr);
    }
    if (lane < nr) u[lane * ldu + i] = make_double2((double)sx, (double)sy);
  }
}

// Eight right-hand sides in FP32 (32 channels): a half-warp per basis
// function, two per warp, each lane holding two adjacent channels (one 16-byte
// load per grid point).  RWG: lanes 0..11 cover the 24 vector channels;
// triangle: four entries at a time, four lanes each over the 8 charge channels.
// Entries run in one flat loop with the grid offset advanced incrementally, so
// the two halves stay in step and each has its own loads in flight.
__global__ void __launch_bounds__(256) k_interp8(const float* __restrict__ mr, const int32_t* __restrict__ mr_base,
                                                 const int32_t* __restrict__ mr_ext,
                                                 const int64_t* __restrict__ mr_off,
                                                 const int32_t* __restrict__ rwg_box, int64_t N,
                                                 const float* __restrict__ mt, const int32_t* __restrict__ mt_base,
                                                 const int32_t* __restrict__ mt_ext,
                                                 const int64_t* __restrict__ mt_off,
                                                 const int32_t* __restrict__ tri_box, int64_t Nt,
                                                 const float2* __restrict__ rg, int sp,
                                                 double2* __restrict__ yA, int64_t ldy, double2* __restrict__ u,
                                                 int64_t ldu) {
  constexpr int C = 32;
  const int lane = threadIdx.x & 31, hl = lane & 15;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 4;  // one basis function per half-warp
  const bool valid = w < N + Nt;
  const int npts = sp * sp * sp;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  const bool is_rwg = valid && w < N;
  const int64_t i = is_rwg ? w : w - N;
  const int32_t* base = is_rwg ? mr_base : mt_base;
  const int32_t* ext = is_rwg ? mr_ext : mt_ext;
  int b0 = 0, b1 = 0, b2 = 0, e0 = 0, e1 = 0, e2 = 0;
  if (valid) {
    b0 = base[3 * i], b1 = base[3 * i + 1], b2 = base[3 * i + 2];
    e0 = ext[3 * i], e1 = ext[3 * i + 1], e2 = ext[3 * i + 2];
  }
  const int ne = e0 * e1 * e2;
  if (is_rwg) {
    const bool act = hl < 12;
    const int d = hl >> 2;
    const float* m = mr + mr_off[i] + d;
    const float2* gp = rg + (int64_t)rwg_box[i] * npts * C + 2 * (act ? hl : 0);
    int64_t off = (int64_t)((b0 * sp + b1) * sp + b2) * C;
    int a1 = 0, a2 = 0;
    for (int e = 0; e < ne; ++e) {
      if (act) {
        const float mv = m[3 * e];
        const float4 g = *reinterpret_cast<const float4*>(gp + off);
        acc.x = fmaf(mv, g.x, acc.x);
        acc.y = fmaf(mv, g.y, acc.y);
        acc.z = fmaf(mv, g.z, acc.z);
        acc.w = fmaf(mv, g.w, acc.w);
      }
      off += C;
      if (++a2 == e2) {
        a2 = 0;
        off += (int64_t)(sp - e2) * C;
        if (++a1 == e1) {
          a1 = 0;
          off += (int64_t)(sp - e1) * sp * C;
        }
      }
    }
  } else if (valid) {
    const int slot = hl >> 2, pr = hl & 3;
    const float* m = mt + mt_off[i];
    const float2* gp = rg + (int64_t)tri_box[i] * npts * C + 24 + 2 * pr;
    if (ne > 0) {
      int e = slot;
      int a0 = e / (e1 * e2), a1 = (e / e2) % e1, a2 = e % e2;
      for (; e < ne; e += 4) {
        const float4 g =
            *reinterpret_cast<const float4*>(gp + (int64_t)(((b0 + a0) * sp + b1 + a1) * sp + b2 + a2) * C);
        const float mv = m[e];
        acc.x = fmaf(mv, g.x, acc.x);
        acc.y = fmaf(mv, g.y, acc.y);
        acc.z = fmaf(mv, g.z, acc.z);
        acc.w = fmaf(mv, g.w, acc.w);
        a2 += 4;
        while (a2 >= e2) {
          a2 -= e2;
          if (++a1 == e1) {
            a1 = 0;
            ++a0;
          }
        }
      }
    }
  }
  // lanes hl < 4 sum lanes hl, hl+4, hl+8, hl+12 of their half-warp: the
  // three components of an RWG (lanes 12..15 hold zeros) or the four entry
  // slots of a triangle
  float4 t;
  t.x = __shfl_down_sync(0xffffffffu, acc.x, 4, 16);
  t.y = __shfl_down_sync(0xffffffffu, acc.y, 4, 16);
  t.z = __shfl_down_sync(0xffffffffu, acc.z, 4, 16);
  t.w = __shfl_down_sync(0xffffffffu, acc.w, 4, 16);
  float4 v = make_float4(acc.x + t.x, acc.y + t.y, acc.z + t.z, acc.w + t.w);
  t.x = __shfl_down_sync(0xffffffffu, v.x, 8, 16);
  t.y = __shfl_down_sync(0xffffffffu, v.y, 8, 16);
  t.z = __shfl_down_sync(0xffffffffu, v.z, 8, 16);
  t.w = __shfl_down_sync(0xffffffffu, v.w, 8, 16);
  v = make_float4(v.x + t.x, v.y + t.y, v.z + t.z, v.w + t.w);
  if (valid && hl < 4) {
    double2* out = is_rwg ? yA : u;
    const int64_t ld = is_rwg ? ldy : ldu;
    out[(int64_t)(2 * hl) * ld + i] = make_double2((double)v.x, (double)v.y);
    out[(int64_t)(2 * hl + 1) * ld + i] = make_double2((double)v.z, (double)v.w);
  }
}

template <typename R>
void launch_interp(const R* mr, const int32_t* mr_base, const int32_t* mr_ext, const int64_t* mr_off,
                   const int32_t* rwg_box, int64_t N, const R* mt, const int32_t* mt_base,
                   const int32_t* mt_ext, const int64_t* mt_off, const int32_t* tri_box, int64_t Nt,
                   const cpx_t<R>* r, int sp, int nr, double2* yA, int64_t ldy, double2* u,
                   int64_t ldu, cudaStream_t s) {
  // nr <= 8 (the far pipeline runs right-hand sides in chunks of at most 8)
  if constexpr (sizeof(R) == 4) {
    if (nr == 8) {
      const int64_t halves = N + Nt;
      k_interp8<<<(unsigned)ceil_div(halves * 16, 256), 256, 0, s>>>(
          (const float*)mr, mr_base, mr_ext, mr_off, rwg_box, N, (const float*)mt, mt_base, mt_ext, mt_off, tri_box,
          Nt, (const float2*)r, sp, yA, ldy, u, ldu);
      return;
    }
  }
  int64_t warps = N + Nt;
  int64_t blocks = ceil_div(warps * 32, 256);
  k_interp<R><<<(unsigned)blocks, 256, 0, s>>>(mr, mr_base, mr_ext, mr_off, rwg_box, N, mt, mt_base, mt_ext,
                                               mt_off, tri_box, Nt, r, sp, nr, yA, ldy, u, ldu);
}

// ---------------------------------------------------------------- translation MAC
// Rh[f][x][c] = sum_{y in IL(x)} Kh[f][off(x - y)] * Qh[f][y][c].
// Tiles group targets that share one source list (the children of a parent
// box on interaction-list levels, chunks of boxes on the top grid level);
// kidx[tile][j][a] holds the offset id of (target a, source j) or -1.  Each
// thread keeps XR targets x CR channels of one frequency in registers, so every
// loaded spectrum value feeds XR complex MACs and every kernel value CR.
// grid: (tile, frequency chunk); block: fpb frequencies x ntx target groups x
// C/CR channel groups.
template <typename R, int XR, int CR>
__global__ void k_mac_tiled(const cpx_t<R>* __restrict__ Qh, cpx_t<R>* __restrict__ Rh,
                            const cpx_t<R>* __restrict__ Kh, int64_t B, int C, int64_t O, int64_t nf,
                            const int64_t* __restrict__ tgt_ptr, const int32_t* __restrict__ tgt,
                            const int64_t* __restrict__ src_ptr, const int32_t* __restrict__ src,
                            const int64_t* __restrict__ kidx_off, const int32_t* __restrict__ kidx,
                            int fpb, int ntx, int64_t f0) {
  using T = cpx_t<R>;
  const int tile = blockIdx.x;
  const int ncg = C / CR;
  const int per_f = ntx * ncg;
  const int fl = threadIdx.x / per_f;
  const int rem = threadIdx.x - fl * per_f;
  const int tg = rem / ncg, cg = rem - (rem / ncg) * ncg;
  const int64_t f = f0 + (int64_t)blockIdx.y * fpb + fl;
  if (fl >= fpb || f >= nf) return;
  const int64_t t0 = tgt_ptr[tile], nt = tgt_ptr[tile + 1] - t0;
  const int64_t s0 = src_ptr[tile], ns = src_ptr[tile + 1] - s0;
  const int xb = tg * XR;
  if (xb >= nt) return;
  const int tpad = (int)(((nt + XR - 1) / XR) * XR);
  const int32_t* kb = kidx + kidx_off[tile] + xb;
  const T* Qf = Qh + f * B * C + cg * CR;
  const T* Kf = Kh + f * O;
  T acc[XR][CR];
#pragma unroll
  for (int a = 0; a < XR; ++a)
#pragma unroll
    for (int c = 0; c < CR; ++c) acc[a][c] = mk<R>(0, 0);
#pragma unroll 2
  for (int64_t j = 0; j < ns; ++j) {
    const int32_t y = __ldg(src + s0 + j);
    T q[CR];
#pragma unroll
    for (int c = 0; c < CR; ++c) q[c] = Qf[(int64_t)y * C + c];
    const int32_t* kr = kb + j * tpad;
#pragma unroll
    for (int a = 0; a < XR; ++a) {
      const int32_t id = __ldg(kr + a);
      if (id < 0) continue;
      const T kv = Kf[id];
#pragma unroll
      for (int c = 0; c < CR; ++c) cfma(acc[a][c], kv, q[c]);
    }
  }
#pragma unroll
  for (int a = 0; a < XR; ++a) {
    if (xb + a >= nt) break;
    T* out = Rh + f * B * C + (int64_t)tgt[t0 + xb + a] * C + cg * CR;
#pragma unroll
    for (int c = 0; c < CR; ++c) out[c] = acc[a][c];
  }
}

// Top grid level, 32 channels (8 right-hand sides), FP32: every block owns one
// tile of <= 128 targets and one frequency; chunks of YS sources are staged in
// shared memory by cp.async (kernel values gathered through the index tile,
// zero-filled for excluded pairs; spectra copied 16 bytes at a time), double
// buffered so the next chunk's gathers run while the current chunk is
// multiplied; each thread runs 8 targets x 4 channels out of shared memory.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  const int sz = valid ? 8 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(sz));
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  const int sz = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(sz));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

template <int YS>
__global__ void __launch_bounds__(128) k_mac_top32(const float2* __restrict__ Qh, float2* __restrict__ Rh,
                                                   const float2* __restrict__ Kh, int64_t B, int64_t O,
                                                   int64_t nf, const int64_t* __restrict__ tgt_ptr,
                                                   const int32_t* __restrict__ tgt,
                                                   const int64_t* __restrict__ src_ptr,
                                                   const int32_t* __restrict__ src,
                                                   const int64_t* __restrict__ kidx_off,
                                                   const int32_t* __restrict__ kidx, int64_t f0) {
  extern __shared__ __align__(16) unsigned char mac_smem[];
  float2(*Ks)[YS][128] = reinterpret_cast<float2(*)[YS][128]>(mac_smem);
  float2(*Qs)[YS][32] = reinterpret_cast<float2(*)[YS][32]>(mac_smem + 2 * sizeof(float2) * YS * 128);
  const int tile = blockIdx.x;
  const int64_t f = f0 + blockIdx.y;
  if (f >= nf) return;
  const int64_t t0 = tgt_ptr[tile], nt = tgt_ptr[tile + 1] - t0;
  const int64_t s0 = src_ptr[tile], ns = src_ptr[tile + 1] - s0;
  const int tpad = (int)(((nt + 7) / 8) * 8);
  const int32_t* kb = kidx + kidx_off[tile];
  const float2* Qf = Qh + f * B * 32;
  const float2* Kf = Kh + f * O;
  const int tg = threadIdx.x >> 3, cg = threadIdx.x & 7;
  const float2 zero = make_float2(0.f, 0.f);
  auto stage = [&](int buf, int64_t j0) {
    const int jn = (int)min((int64_t)YS, ns - j0);
    for (int e = threadIdx.x; e < YS * 128; e += 128) {
      const int j = e >> 7, a = e & 127;
      int32_t id = -1;
      if (j < jn && a < tpad) id = __ldg(kb + (j0 + j) * tpad + a);
      cp_async8(&Ks[buf][j][a], id >= 0 ? (const void*)(Kf + id) : (const void*)Kf, id >= 0);
    }
    for (int e = threadIdx.x; e < YS * 16; e += 128) {
      const int j = e >> 4, c2 = (e & 15) * 2;
      const bool ok = j < jn;
      const int32_t y = ok ? __ldg(src + s0 + j0 + j) : 0;
      cp_async16(&Qs[buf][j][c2], Qf + (int64_t)y * 32 + c2, ok);
    }
    cp_async_commit();
  };
  float2 acc[8][4];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = zero;
  const int nchunks = (int)((ns + YS - 1) / YS);
  if (nchunks > 0) stage(0, 0);
  for (int ch = 0; ch < nchunks; ++ch) {
    const int buf = ch & 1;
    if (ch + 1 < nchunks) {
      stage(buf ^ 1, (int64_t)(ch + 1) * YS);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const int jn = (int)min((int64_t)YS, ns - (int64_t)ch * YS);
    if (tg * 8 < nt) {
      for (int j = 0; j < jn; ++j) {
        const float4 qa = *reinterpret_cast<const float4*>(&Qs[buf][j][cg * 4]);
        const float4 qb = *reinterpret_cast<const float4*>(&Qs[buf][j][cg * 4 + 2]);
        const float2 q[4] = {make_float2(qa.x, qa.y), make_float2(qa.z, qa.w), make_float2(qb.x, qb.y),
                             make_float2(qb.z, qb.w)};
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          const float2 kv = Ks[buf][j][tg * 8 + a];
#pragma unroll
          for (int c = 0; c < 4; ++c) cfma(acc[a][c], kv, q[c]);
        }
      }
    }
    __syncthreads();
  }
  if (tg * 8 >= nt) return;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    if (tg * 8 + a >= nt) break;
    float2* out = Rh + f * B * 32 + (int64_t)tgt[t0 + tg * 8 + a] * 32 + cg * 4;
    *reinterpret_cast<float4*>(out) = make_float4(acc[a][0].x, acc[a][0].y, acc[a][1].x, acc[a][1].y);
    *reinterpret_cast<float4*>(out + 2) = make_float4(acc[a][2].x, acc[a][2].y, acc[a][3].x, acc[a][3].y);
  }
}

// Interaction-list levels, FP32: the kernel values of one frequency are at most
// O (<= 316 on these levels) complex numbers; every block stages the rows of its
// fpb frequencies in shared memory, so the per-pair kernel lookups hit shared
// memory and only the spectra come from L1/L2.
template <int XR, int CR>
__global__ void __launch_bounds__(128) k_mac_il32(const float2* __restrict__ Qh, float2* __restrict__ Rh,
                                                  const float2* __restrict__ Kh, int64_t B, int C, int64_t O,
                                                  int64_t nf, const int64_t* __restrict__ tgt_ptr,
                                                  const int32_t* __restrict__ tgt,
                                                  const int64_t* __restrict__ src_ptr,
                                                  const int32_t* __restrict__ src,
                                                  const int64_t* __restrict__ kidx_off,
                                                  const int32_t* __restrict__ kidx, int fpb, int64_t f0) {
  extern __shared__ __align__(16) unsigned char mac_smem[];
  float2* Kr = reinterpret_cast<float2*>(mac_smem);   // [fpb][O]
  const int tile = blockIdx.x;
  const int64_t fb = f0 + (int64_t)blockIdx.y * fpb;
  for (int e = threadIdx.x; e < fpb * O; e += blockDim.x) {
    const int fl = e / (int)O;
    const int64_t f = fb + fl;
    Kr[e] = f < nf ? __ldg(Kh + f * O + (e - fl * O)) : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int ncg = C / CR;
  const int fl = threadIdx.x / ncg, cg = threadIdx.x - fl * ncg;
  const int64_t f = fb + fl;
  if (fl >= fpb || f >= nf) return;
  const int64_t t0 = tgt_ptr[tile], nt = tgt_ptr[tile + 1] - t0;
  const int64_t s0 = src_ptr[tile], ns = src_ptr[tile + 1] - s0;
  const int32_t* kb = kidx + kidx_off[tile];
  const float2* Qf = Qh + f * B * C + cg * CR;
  const float2* Kf = Kr + fl * O;
  float2 acc[XR][CR];
#pragma unroll
  for (int a = 0; a < XR; ++a)
#pragma unroll
    for (int c = 0; c < CR; ++c) acc[a][c] = make_float2(0.f, 0.f);
  for (int64_t j = 0; j < ns; ++j) {
    const int32_t y = __ldg(src + s0 + j);
    float2 q[CR];
#pragma unroll
    for (int c2 = 0; c2 < CR; c2 += 2) {
      const float4 qa = __ldg(reinterpret_cast<const float4*>(Qf + (int64_t)y * C + c2));
      q[c2] = make_float2(qa.x, qa.y);
      q[c2 + 1] = make_float2(qa.z, qa.w);
    }
    const int4 ia = __ldg(reinterpret_cast<const int4*>(kb + j * XR));
    const int4 ib = __ldg(reinterpret_cast<const int4*>(kb + j * XR + 4));
    const int ids[8] = {ia.x, ia.y, ia.z, ia.w, ib.x, ib.y, ib.z, ib.w};
#pragma unroll
    for (int a = 0; a < XR; ++a) {
      if (ids[a] < 0) continue;
      const float2 kv = Kf[ids[a]];
#pragma unroll
      for (int c = 0; c < CR; ++c) cfma(acc[a][c], kv, q[c]);
    }
  }
#pragma unroll
  for (int a = 0; a < XR; ++a) {
    if (a >= nt) break;
    float2* out = Rh + f * B * C + (int64_t)tgt[t0 + a] * C + cg * CR;
#pragma unroll
    for (int c2 = 0; c2 < CR; c2 += 2)
      *reinterpret_cast<float4*>(out + c2) =
          make_float4(acc[a][c2].x, acc[a][c2].y, acc[a][c2 + 1].x, acc[a][c2 + 1].y);
  }
}

template <typename R>
void launch_mac(const cpx_t<R>* Qh, cpx_t<R>* Rh, const cpx_t<R>* Kh, int64_t B, int C, int64_t O,
                int64_t nf, int64_t ntiles, int max_tile_targets, const int64_t* tgt_ptr, const int32_t* tgt,
                const int64_t* src_ptr, const int32_t* src, const int64_t* kidx_off, const int32_t* kidx,
                cudaStream_t s) {
  if (B <= 0 || nf <= 0 || ntiles <= 0) return;
  // a negative tile size asks for the register-tile kernel (autotuner choice)
  const bool force_reg = max_tile_targets < 0;
  if (force_reg) max_tile_targets = -max_tile_targets;
  if (!force_reg && sizeof(R) == 4 && C == 32 && max_tile_targets > 8 && max_tile_targets <= 128) {
    constexpr int YS = 16;
    const size_t smem = 2 * sizeof(float2) * YS * (128 + 32);
    static SmemAttr attr;
    smem_attr_once(k_mac_top32<YS>, (int)smem, attr.v);
    for (int64_t f0 = 0; f0 < nf; f0 += 65535) {
      int64_t nfc = std::min<int64_t>(65535, nf - f0);
      dim3 grid((unsigned)ntiles, (unsigned)nfc);
      k_mac_top32<YS><<<grid, 128, smem, s>>>((const float2*)Qh, (float2*)Rh, (const float2*)Kh, B, O, nf, tgt_ptr,
                                              tgt, src_ptr, src, kidx_off, kidx, f0);
    }
    return;
  }
  if (!force_reg && sizeof(R) == 4 && (C % 2) == 0 && C >= 16 && max_tile_targets <= 8 && O <= 2048) {
    // interaction-list tiles (<= 8 targets): kernel rows of fpb frequencies in
    // shared memory; CRI channels per thread (2: fewer registers, more warps
    // in flight for this latency-bound loop)
    constexpr int CRI = 2;
    const int ncg = C / CRI;
    int fpb = 128 / ncg;
    if (fpb < 1) fpb = 1;
    while (fpb > 1 && (size_t)fpb * O * sizeof(float2) > 64 * 1024) fpb >>= 1;
    const size_t smem = (size_t)fpb * O * sizeof(float2);
    static SmemAttr attr;
    smem_attr_once(k_mac_il32<8, CRI>, 64 * 1024, attr.v);
    const int64_t fchunk = (int64_t)65535 * fpb;
    for (int64_t f0 = 0; f0 < nf; f0 += fchunk) {
      int64_t nfc = std::min<int64_t>(fchunk, nf - f0);
      dim3 grid((unsigned)ntiles, (unsigned)ceil_div(nfc, fpb));
      k_mac_il32<8, CRI><<<grid, fpb * ncg, smem, s>>>((const float2*)Qh, (float2*)Rh, (const float2*)Kh, B, C, O,
                                                       nf, tgt_ptr, tgt, src_ptr, src, kidx_off, kidx, fpb, f0);
    }
    return;
  }
  constexpr int XR = 8, CR = 4;
  const int ncg = C / CR;
  const int ntx = (max_tile_targets + XR - 1) / XR;
  const int per_f = ntx * ncg;
  int fpb = per_f >= 128 ? 1 : 128 / per_f;
  const int threads = fpb * per_f;
  const int64_t fchunk = (int64_t)65535 * fpb;
  for (int64_t f0 = 0; f0 < nf; f0 += fchunk) {
    int64_t nfc = std::min<int64_t>(fchunk, nf - f0);
    dim3 grid((unsigned)ntiles, (unsigned)ceil_div(nfc, fpb));
    k_mac_tiled<R, XR, CR><<<grid, threads, 0, s>>>(Qh, Rh, Kh, B, C, O, nf, tgt_ptr, tgt, src_ptr, src, kidx_off,
                                                    kidx, fpb, ntx, f0);
  }
}

// ---------------------------------------------------------------- kernel samples
// Kc[o][i0][i1][i2] = g(o h + t Delta), t_d = i_d (i_d < shat) or i_d - n, FP64.
// Samples of the Green's function g(D) = exp(-jkR) / (4 pi R) (comp < 0) or
// of one entry of its Hessian d_a d_b g (comp 0..5: ab = 00, 01, 02, 11, 12,
// 22; the dyadic factorization of Sec. VI-C) at D = o h + t Delta, with
//   d_a d_b g = g2 r_a r_b + (g1 / R) (delta_ab - r_a r_b),
//   g1 = dg/dR = -(jk + 1/R) g,  g2 = d2g/dR2 = ((jk + 1/R)^2 + 1/R^2) g,
// r = D / R.
__global__ void k_kernel_samples(double2* __restrict__ Kc, const int32_t* __restrict__ offsets,
                                 int64_t o0, int64_t no, int n, int shat, double h, double Delta,
                                 double k, int comp) {
  const int64_t n3 = (int64_t)n * n * n;
  const int64_t total = no * n3;
  const int ca = comp < 0 ? 0 : (comp < 3 ? 0 : (comp < 5 ? 1 : 2));
  const int cb = comp < 0 ? 0 : (comp < 3 ? comp : (comp < 5 ? comp - 2 : 2));
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t o = idx / n3, e = idx - o * n3;
    int i0 = (int)(e / (n * n)), i1 = (int)((e / n) % n), i2 = (int)(e % n);
    int t0 = i0 < shat ? i0 : i0 - n, t1 = i1 < shat ? i1 : i1 - n, t2 = i2 < shat ? i2 : i2 - n;
    const int32_t* ov = offsets + 3 * (o0 + o);
    double d[3] = {ov[0] * h + t0 * Delta, ov[1] * h + t1 * Delta, ov[2] * h + t2 * Delta};
    double R = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double sn, cs;
    sincos(k * R, &sn, &cs);
    double fct = 1.0 / (12.566370614359172953850573533118 * R);
    const double2 g = make_double2(cs * fct, -sn * fct);
    if (comp < 0) {
      Kc[idx] = g;
      continue;
    }
    // a = 1/R + jk; g1 = -a g; g2 = (a^2 + 1/R^2) g = (2/R^2 - k^2 + 2jk/R) g
    const double iR = 1.0 / R;
    const double2 a = make_double2(iR, k);
    const double2 g1 = make_double2(-(a.x * g.x - a.y * g.y), -(a.x * g.y + a.y * g.x));
    const double2 c2 = make_double2(2.0 * iR * iR - k * k, 2.0 * k * iR);
    const double2 g2 = make_double2(c2.x * g.x - c2.y * g.y, c2.x * g.y + c2.y * g.x);
    const double rr = d[ca] * d[cb] * iR * iR;
    const double dl = (ca == cb ? 1.0 : 0.0) - rr;
    Kc[idx] = make_double2(g2.x * rr + g1.x * iR * dl, g2.y * rr + g1.y * iR * dl);
  }
}

// Dyadic translation (Sec. VI-C): for every frequency, target box x and
// right-hand side c, R[x][a] = sum_{y in IL(x)} sum_b H_ab(x - y) Q[y][b] over
// the three vector components a, b (H symmetric: six spectra, ab = 00, 01,
// 02, 11, 12, 22); the fourth component of R is set to zero.  Q and R are
// [n^3][B][4 nr] (component-major channels), K[ab] are [n^3][O].  One thread
// per (frequency, box, right-hand side), the interaction lists of the level.
template <typename R>
__global__ void k_mac_dyad(const cpx_t<R>* __restrict__ Q, cpx_t<R>* __restrict__ Rout, KH6<R> K, int64_t B,
                           int nr, int64_t nf, int64_t O, const int64_t* __restrict__ il_ptr,
                           const int32_t* __restrict__ il_src, const int32_t* __restrict__ il_off) {
  using T = cpx_t<R>;
  const int64_t C = 4 * nr;
  const int64_t total = nf * B * nr;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx % nr);
    const int64_t x = (idx / nr) % B, f = idx / (nr * B);
    T acc[3] = {mk<R>(0, 0), mk<R>(0, 0), mk<R>(0, 0)};
    for (int64_t e = il_ptr[x]; e < il_ptr[x + 1]; ++e) {
      const T* q = Q + (f * B + il_src[e]) * C + c;
      const T q0 = q[0], q1 = q[nr], q2 = q[2 * nr];
      const int64_t ko = f * O + il_off[e];
      const T h00 = K.k[0][ko], h01 = K.k[1][ko], h02 = K.k[2][ko];
      const T h11 = K.k[3][ko], h12 = K.k[4][ko], h22 = K.k[5][ko];
      cfma(acc[0], h00, q0);
      cfma(acc[0], h01, q1);
      cfma(acc[0], h02, q2);
      cfma(acc[1], h01, q0);
      cfma(acc[1], h11, q1);
      cfma(acc[1], h12, q2);
      cfma(acc[2], h02, q0);
      cfma(acc[2], h12, q1);
      cfma(acc[2], h22, q2);
    }
    T* r = Rout + (f * B + x) * C + c;
    r[0] = acc[0];
    r[nr] = acc[1];
    r[2 * nr] = acc[2];
    r[3 * nr] = mk<R>(0, 0);
  }
}

template <typename R>
void launch_mac_dyad(const cpx_t<R>* Q, cpx_t<R>* Rout, KH6<R> K, int64_t B, int nr, int64_t nf, int64_t O,
                     const int64_t* il_ptr, const int32_t* il_src, const int32_t* il_off, cudaStream_t s) {
  const int64_t total = nf * B * nr;
  if (total <= 0) return;
  int64_t blocks = ceil_div(total, 256);
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_mac_dyad<R><<<(unsigned)blocks, 256, 0, s>>>(Q, Rout, K, B, nr, nf, O, il_ptr, il_src, il_off);
}
template void launch_mac_dyad<float>(const float2*, float2*, KH6<float>, int64_t, int, int64_t, int64_t,
                                     const int64_t*, const int32_t*, const int32_t*, cudaStream_t);
template void launch_mac_dyad<double>(const double2*, double2*, KH6<double>, int64_t, int, int64_t, int64_t,
                                      const int64_t*, const int32_t*, const int32_t*, cudaStream_t);

void launch_kernel_samples(double2* Kc, const int32_t* offsets, int64_t o0, int64_t no, int n,
                           int shat, double h, double Delta, double k, int comp, cudaStream_t s) {
  int64_t total = no * (int64_t)n * n * n;
  if (total <= 0) return;
  int64_t blocks = ceil_div(total, 256);
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_kernel_samples<<<(unsigned)blocks, 256, 0, s>>>(Kc, offsets, o0, no, n, shat, h, Delta, k, comp);
}

template <typename R>
__global__ void k_convert(const double2* __restrict__ in, cpx_t<R>* __restrict__ out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = mk<R>((R)in[i].x, (R)in[i].y);
}
template <typename R>
void launch_convert(const double2* in, cpx_t<R>* out, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  int64_t blocks = ceil_div(n, 256);
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_convert<R><<<(unsigned)blocks, 256, 0, s>>>(in, out, n);
}

// ---------------------------------------------------------------- vectors
__global__ void k_permute_in(const double2* __restrict__ x, int64_t ldx, const int32_t* __restrict__ perm,
                             int64_t N, int nr, double2* __restrict__ xs) {
  int64_t total = N * nr;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = idx / N, i = idx - r * N;
    xs[r * N + i] = x[r * ldx + perm[i]];
  }
}
void launch_permute_in(const double2* x, int64_t ldx, const int32_t* perm, int64_t N, int nr,
                       double2* xs, cudaStream_t s) {
  int64_t total = N * nr;
  if (total <= 0) return;
  int64_t blocks = ceil_div(total, 256);
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_permute_in<<<(unsigned)blocks, 256, 0, s>>>(x, ldx, perm, N, nr, xs);
}

// rho[r][t] = sum over the 3 RWGs of triangle t of sign * x (Sigma^T x, FP64)
__global__ void k_charges(const double2* __restrict__ xs, int64_t ldx, const int32_t* __restrict__ tri_rwg,
                          const int8_t* __restrict__ tri_sgn, int64_t Nt, int nr, double2* __restrict__ rho,
                          int64_t ldr) {
  int64_t total = Nt * nr;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = idx / Nt, t = idx - r * Nt;
    double2 a = make_double2(0, 0);
    for (int q = 0; q < 3; ++q) {
      int32_t i = tri_rwg[3 * t + q];
      if (i < 0) continue;
      double2 v = xs[r * ldx + i];
      double sg = (double)tri_sgn[3 * t + q];
      a.x += sg * v.x;
      a.y += sg * v.y;
    }
    rho[r * ldr + t] = a;
  }
}
void launch_charges(const double2* xs, int64_t ldx, const int32_t* tri_rwg, const int8_t* tri_sgn,
                    int64_t Nt, int nr, double2* rho, int64_t ldr, cudaStream_t s) {
  int64_t total = Nt * nr;
  if (total <= 0) return;
  int64_t blocks = ceil_div(total, 256);
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_charges<<<(unsigned)blocks, 256, 0, s>>>(xs, ldx, tri_rwg, tri_sgn, Nt, nr, rho, ldr);
}

// y[r][m] = cA * yA[r][i] + cV * (w[r][t+] - w[r][t-]), m = perm[i]; with
// rts null (direct factorization) the scalar part is w[r][i] itself.
// yAn, wn (optional): near-field parts kept apart from the far parts yA, w
__global__ void k_combine(const double2* __restrict__ yA, int64_t ldA, const double2* __restrict__ w,
                          int64_t ldw, const double2* __restrict__ yAn, const double2* __restrict__ wn,
                          const int32_t* __restrict__ perm, const int32_t* __restrict__ rts,
                          int64_t N, int nr, double2 cA, double2 cV, double2* __restrict__ y, int64_t ldy,
                          double2* __restrict__ yAo, double2* __restrict__ yVo) {
  int64_t total = N * nr;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = idx / N, i = idx - r * N;
    double2 a = yA[r * ldA + i];
    double2 v;
    if (rts) {
      // star factorization: the charge part of RWG i is w(c+) - w(c-)
      double2 wp = w[r * ldw + rts[2 * i]], wm = w[r * ldw + rts[2 * i + 1]];
      if (yAn) {
        a = cadd(a, yAn[r * ldA + i]);
        wp = cadd(wp, wn[r * ldw + rts[2 * i]]);
        wm = cadd(wm, wn[r * ldw + rts[2 * i + 1]]);
      }
      v = make_double2(wp.x - wm.x, wp.y - wm.y);
    } else {
      // direct factorization: the scalar part is per RWG already
      v = w[r * ldw + i];
      if (yAn) {
        a = cadd(a, yAn[r * ldA + i]);
        v = cadd(v, wn[r * ldw + i]);
      }
    }
    int64_t m = perm[i];
    if (y) y[r * ldy + m] = cadd(cmul(cA, a), cmul(cV, v));
    if (yAo) yAo[r * ldy + m] = a;
    if (yVo) yVo[r * ldy + m] = v;
  }
}
void launch_combine(const double2* yA, int64_t ldA, const double2* w, int64_t ldw, const double2* yAn,
                    const double2* wn, const int32_t* rwg_perm, const int32_t* rwg_tri_sorted, int64_t N, int nr,
                    double2 cA, double2 cV, double2* y, int64_t ldy, double2* yAout, double2* yVout,
                    cudaStream_t s) {
  int64_t total = N * nr;
  if (total <= 0) return;
  int64_t blocks = ceil_div(total, 256);
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_combine<<<(unsigned)blocks, 256, 0, s>>>(yA, ldA, w, ldw, yAn, wn, rwg_perm, rwg_tri_sorted, N, nr, cA, cV,
                                             y, ldy, yAout, yVout);
}

// Plane-wave RHS: per RWG, both triangles with a degree-10 collapsed rule.
__constant__ double c_q6[3][36];
__global__ void k_rhs_pw(const double* __restrict__ V, const int32_t* __restrict__ T,
                         const double* __restrict__ area, const int32_t* __restrict__ tri_pm,
                         const int32_t* __restrict__ free_pm, int64_t N, double k,
                         const double* __restrict__ khat, const double* __restrict__ pol, int nr,
                         double2* __restrict__ rhs, int64_t ld) {
  int64_t total = N * nr;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = idx / N, m = idx - r * N;
    const double* kh = khat + 3 * r;
    const double* pl = pol + 3 * r;
    double2 acc = make_double2(0, 0);
    for (int s = 0; s < 2; ++s) {
      int t = tri_pm[2 * m + s];
      const double* xf = V + 3 * free_pm[2 * m + s];
      double sc = (s == 0 ? 1.0 : -1.0) / (2.0 * area[t]);
      const double* a = V + 3 * T[3 * t];
      const double* b = V + 3 * T[3 * t + 1];
      const double* c = V + 3 * T[3 * t + 2];
      for (int q = 0; q < 36; ++q) {
        double xi = c_q6[0][q], eta = c_q6[1][q], w = c_q6[2][q] * 2.0 * area[t];
        double x[3];
        for (int d = 0; d < 3; ++d) x[d] = a[d] + xi * (b[d] - a[d]) + eta * (c[d] - a[d]);
        double ph = -k * (kh[0] * x[0] + kh[1] * x[1] + kh[2] * x[2]);
        double sn, cs;
        sincos(ph, &sn, &cs);
        double fp = 0;
        for (int d = 0; d < 3; ++d) fp += (x[d] - xf[d]) * pl[d];
        fp *= sc * w;
        acc.x += fp * cs;
        acc.y += fp * sn;
      }
    }
    rhs[r * ld + m] = acc;
  }
}
int upload_rhs_rule(const double* q6) {
  return cudaMemcpyToSymbol(c_q6, q6, sizeof(double) * 108) == cudaSuccess ? 0 : -1;
}
void launch_rhs_planewave(const double* V, const int32_t* T, const double* area, const int32_t* tri_pm,
                          const int32_t* free_pm, int64_t N, double k, const double* khat,
                          const double* pol, int nr, double2* rhs, int64_t ld, cudaStream_t s) {
  int64_t total = N * nr;
  if (total <= 0) return;
  int64_t blocks = ceil_div(total, 128);
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_rhs_pw<<<(unsigned)blocks, 128, 0, s>>>(V, T, area, tri_pm, free_pm, N, k, khat, pol, nr, rhs, ld);
}

// ---------------------------------------------------------------- Krylov
// Block sum of 512 per-thread values in a fixed order (warp shuffles, then
// the 16 warp sums in ascending order); the result is valid in thread 0.
template <typename T>
__device__ __forceinline__ T block_sum512(T v, T* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  T s = 0;
  if (threadIdx.x == 0)
    for (int i = 0; i < 16; ++i) s += red[i];
  return s;
}

// h[r][i] = sum_n conj(V[r][i][n]) w[r][n]; grid (nbasis, nr), 512 threads.
// One block per output and a fixed summation order: the Arnoldi coefficients,
// and so the iterates, are the same on every run.
__global__ void __launch_bounds__(512) k_multidot(const double2* __restrict__ Vb, int64_t ldv_r, int64_t ldv_i,
                                                  const double2* __restrict__ w, int64_t ldw, int64_t N,
                                                  const int* __restrict__ active, double2* __restrict__ h,
                                                  int nbasis) {
  const int i = blockIdx.x, r = blockIdx.y;
  if (active && !active[r]) {
    if (threadIdx.x == 0) h[(int64_t)r * nbasis + i] = make_double2(0, 0);
    return;
  }
  const double2* v = Vb + r * ldv_r + i * ldv_i;
  const double2* wr = w + r * ldw;
  double sx = 0, sy = 0;
  for (int64_t n = threadIdx.x; n < N; n += blockDim.x) {
    double2 a = v[n], b = wr[n];
    sx += a.x * b.x + a.y * b.y;
    sy += a.x * b.y - a.y * b.x;
  }
  __shared__ double rx[16], ry[16];
  sx = block_sum512(sx, rx);
  sy = block_sum512(sy, ry);
  if (threadIdx.x == 0) h[(int64_t)r * nbasis + i] = make_double2(sx, sy);
}
void launch_multidot(const double2* Vb, int64_t ldv_r, int64_t ldv_i, int nbasis, const double2* w,
                     int64_t ldw, int64_t N, int nr, const int* active, double2* h, cudaStream_t s) {
  if (nbasis <= 0 || nr <= 0) return;
  dim3 grid(nbasis, nr);
  k_multidot<<<grid, 512, 0, s>>>(Vb, ldv_r, ldv_i, w, ldw, N, active, h, nbasis);
}

// w[r][n] += sign * sum_i h[r][i] V[r][i][n]
__global__ void k_multiaxpy(const double2* __restrict__ Vb, int64_t ldv_r, int64_t ldv_i, int nbasis,
                            const double2* __restrict__ h, int hstride, double2* __restrict__ w,
                            int64_t ldw, int64_t N, int nr, const int* __restrict__ active, double sign) {
  int64_t total = N * nr;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = idx / N, n = idx - r * N;
    if (active && !active[r]) continue;
    double2 acc = make_double2(0, 0);
    for (int i = 0; i < nbasis; ++i) cfma(acc, h[r * hstride + i], Vb[r * ldv_r + i * ldv_i + n]);
    double2 t = w[r * ldw + n];
    w[r * ldw + n] = make_double2(t.x + sign * acc.x, t.y + sign * acc.y);
  }
}
void launch_multiaxpy(const double2* Vb, int64_t ldv_r, int64_t ldv_i, int nbasis, const double2* h,
                      int hstride, double2* w, int64_t ldw, int64_t N, int nr, const int* active,
                      double sign, cudaStream_t s) {
  int64_t total = N * nr;
  if (total <= 0 || nbasis <= 0) return;
  int64_t blocks = ceil_div(total, 256);
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_multiaxpy<<<(unsigned)blocks, 256, 0, s>>>(Vb, ldv_r, ldv_i, nbasis, h, hstride, w, ldw, N, nr, active,
                                               sign);
}

// out = a x + b y over n complex entries (real a, b)
__global__ void k_lincomb(const double2* __restrict__ x, const double2* __restrict__ y, double a, double b,
                          double2* __restrict__ out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double2 u = x[i], v = y[i];
    out[i] = make_double2(a * u.x + b * v.x, a * u.y + b * v.y);
  }
}
void launch_lincomb(const double2* x, const double2* y, double a, double b, double2* out, int64_t n,
                    cudaStream_t s) {
  if (n <= 0) return;
  int64_t blocks = ceil_div(n, 256);
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_lincomb<<<(unsigned)blocks, 256, 0, s>>>(x, y, a, b, out, n);
}

// out = a conj(x)
__global__ void k_conj_scale(const double2* __restrict__ x, double a, double2* __restrict__ out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double2 v = x[i];
    out[i] = make_double2(a * v.x, -a * v.y);
  }
}
void launch_conj_scale(const double2* x, double a, double2* out, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  int64_t blocks = ceil_div(n, 256);
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_conj_scale<<<(unsigned)blocks, 256, 0, s>>>(x, a, out, n);
}

// out[r] = sum_n |w[r][n]|^2; one 512-thread block per vector, fixed order
__global__ void __launch_bounds__(512) k_norms(const double2* __restrict__ w, int64_t ldw, int64_t N,
                                               double* out) {
  const int r = blockIdx.x;
  double s = 0;
  for (int64_t n = threadIdx.x; n < N; n += blockDim.x) {
    double2 a = w[r * ldw + n];
    s += a.x * a.x + a.y * a.y;
  }
  __shared__ double red[16];
  s = block_sum512(s, red);
  if (threadIdx.x == 0) out[r] = s;
}
void launch_norms(const double2* w, int64_t ldw, int64_t N, int nr, double* out, cudaStream_t s) {
  if (nr <= 0) return;
  k_norms<<<nr, 512, 0, s>>>(w, ldw, N, out);
}

// explicit instantiations
template void launch_mode_pair<float>(const float2*, View, float2*, View, int64_t, int, int, int, int, int, int,
                                      const float*, const float*, const int64_t*, const int64_t*, const int8_t*,
                                      const int8_t*, cudaStream_t);
template void launch_mode_pair<double>(const double2*, View, double2*, View, int64_t, int, int, int, int, int, int,
                                       const double*, const double*, const int64_t*, const int64_t*,
                                       const int8_t*, const int8_t*, cudaStream_t);
template bool launch_dft<float>(const float2*, View, float2*, View, int64_t, int, int, int, int, int, int,
                                const float2*, int, bool, cudaStream_t);
template bool launch_dft<double>(const double2*, View, double2*, View, int64_t, int, int, int, int, int, int,
                                 const double2*, int, bool, cudaStream_t);
template void launch_mode<float>(const float2*, View, float2*, View, int64_t, int, int, int, int, int, int,
                                 const void*, const void*, bool, const int8_t*, const int64_t*, bool,
                                 cudaStream_t);
template void launch_mode<double>(const double2*, View, double2*, View, int64_t, int, int, int, int, int, int,
                                  const void*, const void*, bool, const int8_t*, const int64_t*, bool,
                                  cudaStream_t);
template void launch_gather_build<float>(const float*, const int32_t*, const int32_t*, const int64_t*,
                                         const float*, const int32_t*, const int32_t*, const int64_t*,
                                         const int64_t*, const int64_t*, int64_t, int, int32_t*, int32_t*, float*,
                                         float*, cudaStream_t);
template void launch_gather_build<double>(const double*, const int32_t*, const int32_t*, const int64_t*,
                                          const double*, const int32_t*, const int32_t*, const int64_t*,
                                          const int64_t*, const int64_t*, int64_t, int, int32_t*, int32_t*,
                                          double*, double*, cudaStream_t);
template void launch_anterp<float>(const float*, const float*, const int32_t*, const int32_t*, const int64_t*,
                                   const int64_t*, const int64_t*, const int64_t*, int64_t, const int32_t*,
                                   const float2*, int64_t, const float2*, int64_t, int, float2*, int, cudaStream_t);
template void launch_anterp<double>(const double*, const double*, const int32_t*, const int32_t*, const int64_t*,
                                    const int64_t*, const int64_t*, const int64_t*, int64_t, const int32_t*,
                                    const double2*, int64_t, const double2*, int64_t, int, double2*, int,
                                    cudaStream_t);
template void launch_interp<float>(const float*, const int32_t*, const int32_t*, const int64_t*, const int32_t*,
                                   int64_t, const float*, const int32_t*, const int32_t*, const int64_t*,
                                   const int32_t*, int64_t, const float2*, int, int, double2*, int64_t,
                                   double2*, int64_t, cudaStream_t);
template void launch_interp<double>(const double*, const int32_t*, const int32_t*, const int64_t*,
                                    const int32_t*, int64_t, const double*, const int32_t*, const int32_t*,
                                    const int64_t*, const int32_t*, int64_t, const double2*, int, int,
                                    double2*, int64_t, double2*, int64_t, cudaStream_t);
template void launch_mac<float>(const float2*, float2*, const float2*, int64_t, int, int64_t, int64_t, int64_t,
                                int, const int64_t*, const int32_t*, const int64_t*, const int32_t*,
                                const int64_t*, const int32_t*, cudaStream_t);
template void launch_mac<double>(const double2*, double2*, const double2*, int64_t, int, int64_t, int64_t,
                                 int64_t, int, const int64_t*, const int32_t*, const int64_t*, const int32_t*,
                                 const int64_t*, const int32_t*, cudaStream_t);
template void launch_convert<float>(const double2*, float2*, int64_t, cudaStream_t);
template void launch_convert<double>(const double2*, double2*, int64_t, cudaStream_t);

}  // namespace efie
