// Learned mesh-local preconditioner (not part of the paper): a message-passing
// network on the RWG adjacency graph mapping a residual r to an approximate
// error z ~ T^-1 r, used as the flexible right preconditioner of FGMRES.
//
//   s = rms(r), x = [Re r/s, Im r/s, l/mean(l), 1]
//   h = tanh(x We^T + be)
//   3 x: a = sum_n s_mn h_n ;  h = tanh([h | a] [Ws | Wn]^T + bl) + h
//   z = s ((h Wd^T + bd)_0 + j (h Wd^T + bd)_1)
//
// Width 64.  Weights are kept in FP32 (Adam state) and used as bfloat16; every
// matrix product takes bfloat16 operands and accumulates in FP32 on the tensor
// cores (mma m16n8k16, 64-node tiles staged in shared memory).  Training runs
// the hand-written backward kernels below and Adam on the GPU.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cstdint>
#include <random>
#include <vector>

#include "common.cuh"
#include "device_api.cuh"
#include "plan.hpp"

namespace efie {

constexpr int NW = 64;       // width
constexpr int NL = 3;        // message-passing layers
constexpr int NIN = 4;       // input features
constexpr int TILE = 64;     // nodes per block
constexpr int KP = 128 + 8;  // padded row (bf16) of the [h | a] tile

// parameter offsets in the flat FP32 vector (same order as the reference)
constexpr int OFF_WE = 0;
constexpr int OFF_BE = OFF_WE + NW * NIN;
constexpr int LAYER_SZ = NW * NW * 2 + NW;
constexpr int OFF_L0 = OFF_BE + NW;
constexpr int OFF_WD = OFF_L0 + NL * LAYER_SZ;
constexpr int OFF_BD = OFF_WD + 2 * NW;
constexpr int NPARAM = OFF_BD + 2;
// Gradient reductions are deterministic: each kernel runs on a fixed number of
// blocks (a function of N only), every block writes its partial sums in a
// fixed order, and k_nn_reduce adds the partials block by block.  Training
// from a seed therefore gives the same network on every run.
constexpr int NB_RED = 256;                    // blocks of the reducing kernels
constexpr int PART_W = 2 * NW * NW + NW;       // widest partial: one layer's dWs | dWn | dbias

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ float bf16r(float a) { return __bfloat162float(__float2bfloat16_rn(a)); }

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// A fragment (16 x 16, row-major in smem with row stride ld bf16)
__device__ __forceinline__ void load_a(const __nv_bfloat16* A, int ld, int r0, int k0, uint32_t* a) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  a[0] = *reinterpret_cast<const uint32_t*>(A + (r0 + g) * ld + k0 + 2 * t);
  a[1] = *reinterpret_cast<const uint32_t*>(A + (r0 + g + 8) * ld + k0 + 2 * t);
  a[2] = *reinterpret_cast<const uint32_t*>(A + (r0 + g) * ld + k0 + 8 + 2 * t);
  a[3] = *reinterpret_cast<const uint32_t*>(A + (r0 + g + 8) * ld + k0 + 8 + 2 * t);
}
// B fragment (16 x 8) from Bt stored [n][k] row-major (stride ld): B[k][n] = Bt[n][k]
__device__ __forceinline__ void load_b(const __nv_bfloat16* Bt, int ld, int n0, int k0, uint32_t* b) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  b[0] = *reinterpret_cast<const uint32_t*>(Bt + (n0 + g) * ld + k0 + 2 * t);
  b[1] = *reinterpret_cast<const uint32_t*>(Bt + (n0 + g) * ld + k0 + 8 + 2 * t);
}

// ----------------------------------------------------------------- forward
// s^2 = mean |r|^2 (sum computed by the caller), then encoder
__global__ void k_nn_encode(const double2* __restrict__ r, const float* __restrict__ lnorm, int64_t N,
                            const double* __restrict__ sumsq, const float* __restrict__ P,
                            float* __restrict__ x_out, float* __restrict__ u0, float* __restrict__ h0) {
  const double s2 = sumsq[0] / (double)N;
  const float inv = s2 > 0 ? (float)(1.0 / sqrt(s2)) : 0.f;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < N * NW;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = idx / NW;
    const int j = (int)(idx - m * NW);
    const double2 v = r[m];
    float x[NIN] = {bf16r((float)v.x * inv), bf16r((float)v.y * inv), bf16r(lnorm[m]), 1.f};
    float u = P[OFF_BE + j];
#pragma unroll
    for (int i = 0; i < NIN; ++i) u = fmaf(x[i], bf16r(P[OFF_WE + j * NIN + i]), u);
    if (u0) u0[idx] = u;
    h0[idx] = tanhf(u);
    if (x_out && j < NIN) x_out[m * NIN + j] = x[j];
  }
}

// One message-passing layer on a tile of 64 nodes:
//   a = sum_n s_mn h_n ; u = [bf16(h) | bf16(a)] Wcat^T + b ; h_out = tanh(u) + h
__global__ void __launch_bounds__(128) k_nn_layer(const float* __restrict__ h, const int32_t* __restrict__ nbr,
                                                  const float* __restrict__ sgn, int64_t N,
                                                  const __nv_bfloat16* __restrict__ Wcat,
                                                  const float* __restrict__ bias, float* __restrict__ h_out,
                                                  float* __restrict__ u_out, float* __restrict__ a_out) {
  __shared__ __align__(16) __nv_bfloat16 Xs[TILE * KP];
  __shared__ __align__(16) __nv_bfloat16 Ws[NW * KP];
  const int64_t m0 = (int64_t)blockIdx.x * TILE;
  for (int i = threadIdx.x; i < NW * 128; i += blockDim.x) Ws[(i >> 7) * KP + (i & 127)] = Wcat[i];
  for (int i = threadIdx.x; i < TILE * NW; i += blockDim.x) {
    const int ml = i >> 6, j = i & 63;
    const int64_t m = m0 + ml;
    float hv = 0.f, av = 0.f;
    if (m < N) {
      hv = h[m * NW + j];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int32_t n = nbr[m * 4 + q];
        if (n >= 0) av = fmaf(sgn[m * 4 + q], h[(int64_t)n * NW + j], av);
      }
      if (a_out) a_out[m * NW + j] = av;
    }
    Xs[ml * KP + j] = __float2bfloat16_rn(hv);
    Xs[ml * KP + 64 + j] = __float2bfloat16_rn(av);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int r0 = warp * 16;
  float acc[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[nt][i] = 0.f;
#pragma unroll
  for (int kt = 0; kt < 8; ++kt) {
    uint32_t a[4];
    load_a(Xs, KP, r0, kt * 16, a);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      uint32_t b[2];
      load_b(Ws, KP, nt * 8, kt * 16, b);
      mma_bf16(acc[nt], a, b);
    }
  }
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int row = r0 + g + (i >= 2 ? 8 : 0);
      const int col = nt * 8 + 2 * t + (i & 1);
      const int64_t m = m0 + row;
      if (m >= N) continue;
      const float u = acc[nt][i] + bias[col];
      if (u_out) u_out[m * NW + col] = u;
      h_out[m * NW + col] = tanhf(u) + h[m * NW + col];
    }
}

// z = s (y0 + j y1), y = bf16(h) Wd^T + bd (one warp per node)
__global__ void k_nn_decode(const float* __restrict__ h, int64_t N, const float* __restrict__ P,
                            const double* __restrict__ sumsq, double2* __restrict__ z) {
  const double s = sqrt(sumsq[0] / (double)N);
  const int lane = threadIdx.x & 31;
  for (int64_t m = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; m < N;
       m += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    float y0 = 0.f, y1 = 0.f;
    for (int j = lane; j < NW; j += 32) {
      const float hv = bf16r(h[m * NW + j]);
      y0 = fmaf(hv, bf16r(P[OFF_WD + j]), y0);
      y1 = fmaf(hv, bf16r(P[OFF_WD + NW + j]), y1);
    }
    for (int o = 16; o > 0; o >>= 1) {
      y0 += __shfl_down_sync(0xffffffffu, y0, o);
      y1 += __shfl_down_sync(0xffffffffu, y1, o);
    }
    if (lane == 0) z[m] = make_double2(s * (double)(y0 + P[OFF_BD]), s * (double)(y1 + P[OFF_BD + 1]));
  }
}

// ----------------------------------------------------------------- backward
// loss terms: sum |z - e|^2 and sum |e|^2, one partial pair per block
// (256 threads), reduced by k_nn_loss_reduce in block order
__global__ void __launch_bounds__(256) k_nn_loss(const double2* __restrict__ z, const double2* __restrict__ e,
                                                 int64_t N, double* __restrict__ dpart) {
  double a = 0, b = 0;
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < N; m += (int64_t)gridDim.x * blockDim.x) {
    const double dx = z[m].x - e[m].x, dy = z[m].y - e[m].y;
    a += dx * dx + dy * dy;
    b += e[m].x * e[m].x + e[m].y * e[m].y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  __shared__ double ra[8], rb[8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    ra[w] = a;
    rb[w] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0, sb = 0;
    for (int i = 0; i < 8; ++i) {
      sa += ra[i];
      sb += rb[i];
    }
    dpart[2 * blockIdx.x] = sa;
    dpart[2 * blockIdx.x + 1] = sb;
  }
}
__global__ void k_nn_loss_reduce(const double* __restrict__ dpart, int nb, double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double a = 0, b = 0;
  for (int i = 0; i < nb; ++i) {
    a += dpart[2 * i];
    b += dpart[2 * i + 1];
  }
  out[0] = a;
  out[1] = b;
}

// G[i] += sum_b part[b][i], b ascending
__global__ void k_nn_reduce(const float* __restrict__ part, int nb, int width, float* __restrict__ G) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= width) return;
  float acc = 0.f;
  for (int b = 0; b < nb; ++b) acc += part[(int64_t)b * width + i];
  G[i] += acc;
}

// g = 2 (z - e) / |e|^2, the gradient of the error loss with respect to z
__global__ void k_nn_err_grad(const double2* __restrict__ z, const double2* __restrict__ e, int64_t N,
                              const double* __restrict__ lossacc, double2* __restrict__ g) {
  const double E = lossacc[1];
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < N; m += (int64_t)gridDim.x * blockDim.x)
    g[m] = make_double2(2.0 * (z[m].x - e[m].x) / E, 2.0 * (z[m].y - e[m].y) / E);
}

// decoder backward from g = dL/dz (dL/dRe z = Re g, dL/dIm z = Im g):
// dy = s (Re g, Im g) ; dWd, dbd ; dh = dy bf16(Wd).  256 threads = 4 nodes x
// 64 features; the grid stride is a multiple of 64, so a thread keeps one
// feature j and sums its own terms; the 4 threads of a feature are added in a
// fixed order and the block writes part[block][2 NW + 2].
__global__ void __launch_bounds__(256) k_nn_decode_back(const float* __restrict__ h,
                                                        const double2* __restrict__ gz, int64_t N,
                                                        const double* __restrict__ sumsq,
                                                        const float* __restrict__ P, float* __restrict__ part,
                                                        float* __restrict__ dh) {
  const double s = sqrt(sumsq[0] / (double)N);
  __shared__ float red[4][2 * NW + 2];
  const int j = threadIdx.x & (NW - 1), q = threadIdx.x >> 6;
  const float w0 = bf16r(P[OFF_WD + j]), w1 = bf16r(P[OFF_WD + NW + j]);
  float p0 = 0.f, p1 = 0.f, c0 = 0.f, c1 = 0.f;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < N * NW;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = idx / NW;
    const float d0 = (float)(s * gz[m].x);
    const float d1 = (float)(s * gz[m].y);
    const float hv = bf16r(h[idx]);
    p0 += d0 * hv;
    p1 += d1 * hv;
    c0 += d0;
    c1 += d1;
    dh[idx] = d0 * w0 + d1 * w1;
  }
  red[q][j] = p0;
  red[q][NW + j] = p1;
  if (j == 0) {
    red[q][2 * NW] = c0;
    red[q][2 * NW + 1] = c1;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * NW + 2; i += blockDim.x)
    part[(int64_t)blockIdx.x * (2 * NW + 2) + i] = ((red[0][i] + red[1][i]) + red[2][i]) + red[3][i];
}

// du = dh (1 - tanh(u)^2)
__global__ void k_nn_du(const float* __restrict__ dh, const float* __restrict__ u, float* __restrict__ du,
                        int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float t = tanhf(u[i]);
    du[i] = dh[i] * (1.f - t * t);
  }
}

// Layer backward over tiles of 64 nodes (each block takes tiles b, b + grid,
// ... in order):
//   dWcat += du^T [bf16(h) | bf16(a)]   (tensor cores, summed over the block's
//                                        tiles in registers)
//   dbias += sum du
//   dX = bf16(du) Wcat  -> dXh (added to dh_next), dXa (neighbour part, stored)
// The block's dWs | dWn | dbias sums go to part[block][PART_W].
__global__ void __launch_bounds__(128) k_nn_layer_back(const float* __restrict__ du, const float* __restrict__ h,
                                                       const float* __restrict__ a, int64_t N,
                                                       const __nv_bfloat16* __restrict__ WcatT,
                                                       float* __restrict__ part, float* __restrict__ dh_next,
                                                       float* __restrict__ dXa) {
  extern __shared__ __align__(16) unsigned char nn_smem[];
  __nv_bfloat16* duT = (__nv_bfloat16*)nn_smem;             // [n][m]      64 x 72
  __nv_bfloat16* XT = duT + NW * (TILE + 8);                 // [k][m]     128 x 72
  __nv_bfloat16* dus = XT + 128 * (TILE + 8);                // [m][n]      64 x 72
  __nv_bfloat16* Wt = dus + TILE * (NW + 8);                 // WcatT [k][n] 128 x 72
  const int LDT = TILE + 8, LDN = NW + 8;
  for (int i = threadIdx.x; i < 128 * NW; i += blockDim.x) Wt[(i >> 6) * LDN + (i & 63)] = WcatT[i];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float accW[16][4];
#pragma unroll
  for (int nt = 0; nt < 16; ++nt)
#pragma unroll
    for (int i = 0; i < 4; ++i) accW[nt][i] = 0.f;
  float accB = 0.f;
  const int64_t ntiles = (N + TILE - 1) / TILE;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t m0 = tile * TILE;
    __syncthreads();   // the previous tile's shared-memory reads are done
    for (int i = threadIdx.x; i < TILE * NW; i += blockDim.x) {
      const int ml = i >> 6, j = i & 63;
      const int64_t m = m0 + ml;
      float dv = 0.f, hv = 0.f, av = 0.f;
      if (m < N) {
        dv = du[m * NW + j];
        hv = h[m * NW + j];
        av = a[m * NW + j];
      }
      const __nv_bfloat16 db = __float2bfloat16_rn(dv);
      duT[j * LDT + ml] = db;
      dus[ml * LDN + j] = db;
      XT[j * LDT + ml] = __float2bfloat16_rn(hv);
      XT[(64 + j) * LDT + ml] = __float2bfloat16_rn(av);
    }
    __syncthreads();
    // dW tile: rows n in [16 warp, +16), cols k in [0,128), K = 64 nodes
#pragma unroll
    for (int kt = 0; kt < TILE / 16; ++kt) {
      uint32_t af[4];
      load_a(duT, LDT, warp * 16, kt * 16, af);
#pragma unroll
      for (int nt = 0; nt < 16; ++nt) {
        uint32_t bf[2];
        load_b(XT, LDT, nt * 8, kt * 16, bf);
        mma_bf16(accW[nt], af, bf);
      }
    }
    // bias gradient
    if (threadIdx.x < NW)
      for (int ml = 0; ml < TILE; ++ml)
        if (m0 + ml < N) accB += du[(m0 + ml) * NW + threadIdx.x];
    // dX tile: rows m in [16 warp, +16), cols k in [0, 128), K = 64 outputs
    float acc[16][4];
#pragma unroll
    for (int nt = 0; nt < 16; ++nt)
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[nt][i] = 0.f;
#pragma unroll
    for (int kt = 0; kt < NW / 16; ++kt) {
      uint32_t af[4];
      load_a(dus, LDN, warp * 16, kt * 16, af);
#pragma unroll
      for (int nt = 0; nt < 16; ++nt) {
        uint32_t bf[2];
        load_b(Wt, LDN, nt * 8, kt * 16, bf);
        mma_bf16(acc[nt], af, bf);
      }
    }
#pragma unroll
    for (int nt = 0; nt < 16; ++nt)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int ml = warp * 16 + g + (i >= 2 ? 8 : 0);
        const int k = nt * 8 + 2 * t + (i & 1);
        const int64_t m = m0 + ml;
        if (m >= N) continue;
        if (k < 64)
          dh_next[m * NW + k] += acc[nt][i];
        else
          dXa[m * NW + (k - 64)] = acc[nt][i];
      }
  }
  float* pb = part + (int64_t)blockIdx.x * PART_W;
#pragma unroll
  for (int nt = 0; nt < 16; ++nt)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int n = warp * 16 + g + (i >= 2 ? 8 : 0);
      const int k = nt * 8 + 2 * t + (i & 1);
      // layout of one layer's parameters: Ws [64][64], Wn [64][64], bias [64]
      pb[k < 64 ? n * NW + k : NW * NW + n * NW + (k - 64)] = accW[nt][i];
    }
  if (threadIdx.x < NW) pb[2 * NW * NW + threadIdx.x] = accB;
}

// dh_next[m] += sum_n s_mn dXa[n]
__global__ void k_nn_gather_back(const float* __restrict__ dXa, const int32_t* __restrict__ nbr,
                                 const float* __restrict__ sgn, int64_t N, float* __restrict__ dh_next) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < N * NW;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = idx / NW;
    const int j = (int)(idx - m * NW);
    float acc = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int32_t n = nbr[m * 4 + q];
      if (n >= 0) acc = fmaf(sgn[m * 4 + q], dXa[(int64_t)n * NW + j], acc);
    }
    dh_next[idx] += acc;
  }
}

// encoder backward: dWe += du0^T bf16(x), dbe += sum du0.  256 threads = 4
// nodes x 64 features, one feature per thread (the grid stride is a multiple
// of 64); the block writes part[block][NW (NIN + 1)] (dWe [64][4], dbe [64]).
__global__ void __launch_bounds__(256) k_nn_encode_back(const float* __restrict__ du0, const float* __restrict__ x,
                                                        int64_t N, float* __restrict__ part) {
  __shared__ float red[4][NW * (NIN + 1)];
  const int j = threadIdx.x & (NW - 1), q = threadIdx.x >> 6;
  float pw[NIN] = {0.f, 0.f, 0.f, 0.f}, pbias = 0.f;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < N * NW;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = idx / NW;
    const float d = du0[idx];
#pragma unroll
    for (int i = 0; i < NIN; ++i) pw[i] += d * x[m * NIN + i];
    pbias += d;
  }
#pragma unroll
  for (int i = 0; i < NIN; ++i) red[q][j * NIN + i] = pw[i];
  red[q][NW * NIN + j] = pbias;
  __syncthreads();
  for (int i = threadIdx.x; i < NW * (NIN + 1); i += blockDim.x)
    part[(int64_t)blockIdx.x * NW * (NIN + 1) + i] = ((red[0][i] + red[1][i]) + red[2][i]) + red[3][i];
}

// bfloat16 copies of the layer matrices: Wcat [64][128] and WcatT [128][64]
__global__ void k_nn_pack(const float* __restrict__ P, __nv_bfloat16* __restrict__ Wcat,
                          __nv_bfloat16* __restrict__ WcatT) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NL * NW * 128; i += gridDim.x * blockDim.x) {
    const int l = i / (NW * 128), rem = i % (NW * 128), n = rem / 128, k = rem % 128;
    const float* L = P + OFF_L0 + l * LAYER_SZ;
    const float w = k < 64 ? L[n * NW + k] : L[NW * NW + n * NW + (k - 64)];
    const __nv_bfloat16 b = __float2bfloat16_rn(w);
    Wcat[l * NW * 128 + n * 128 + k] = b;
    WcatT[l * NW * 128 + k * NW + n] = b;
  }
}

__global__ void k_adam(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ M,
                       float* __restrict__ V, int n, float lr, float b1, float b2, float eps, float c1, float c2,
                       float gscale) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float g = G[i] * gscale;
    M[i] = b1 * M[i] + (1.f - b1) * g;
    V[i] = b2 * V[i] + (1.f - b2) * g * g;
    P[i] -= lr * (M[i] / c1) / (sqrtf(V[i] / c2) + eps);
  }
}

// ----------------------------------------------------------------- host side
struct Net {
  int64_t N = 0;
  std::vector<float> params;            // host copy (FP32)
  float *P = nullptr, *G = nullptr, *M = nullptr, *V = nullptr;
  __nv_bfloat16 *Wcat = nullptr, *WcatT = nullptr;
  int32_t* nbr = nullptr;
  float *sgn = nullptr, *lnorm = nullptr;
  // activations
  float *x = nullptr, *u0 = nullptr;
  float* h[NL + 1] = {nullptr};
  float* u[NL] = {nullptr};
  float* a[NL] = {nullptr};
  float *dh = nullptr, *du = nullptr, *dXa = nullptr;
  double* red = nullptr;   // [0] sum |r|^2, [1..2] loss terms
  float* part = nullptr;   // [NB_RED][PART_W] per-block gradient partials
  double* dpart = nullptr; // [NB_RED][2] per-block loss partials
  int step = 0;
};

static int64_t grid_for(int64_t n, int block) {
  int64_t b = (n + block - 1) / block;
  return b > 152 * 32 ? 152 * 32 : (b < 1 ? 1 : b);
}

int nn_param_count() { return NPARAM; }
void nn_free(Net& net);
Net* nn_new() { return new Net(); }
void nn_delete(Net* n) {
  if (!n) return;
  nn_free(*n);
  delete n;
}

void nn_init_params(std::vector<float>& p, uint64_t seed) {
  // same scales as the reference initialisation (the draws themselves differ)
  std::mt19937_64 rng(seed);
  std::normal_distribution<float> nd(0.f, 1.f);
  p.assign(NPARAM, 0.f);
  for (int i = 0; i < NW * NIN; ++i) p[OFF_WE + i] = nd(rng) / 2.0f;
  for (int l = 0; l < NL; ++l) {
    float* L = p.data() + OFF_L0 + l * LAYER_SZ;
    for (int i = 0; i < NW * NW; ++i) L[i] = nd(rng) * 0.5f / 8.0f;
    for (int i = 0; i < NW * NW; ++i) L[NW * NW + i] = nd(rng) * 0.25f / 8.0f;
  }
  for (int i = 0; i < 2 * NW; ++i) p[OFF_WD + i] = nd(rng) * 0.1f / 8.0f;
}

// graph: neighbour ids / signs [N][4], normalised edge lengths [N]
void nn_setup(Net& net, int64_t N, const std::vector<int32_t>& nbr, const std::vector<float>& sgn,
              const std::vector<float>& lnorm, const std::vector<float>& params, bool training) {
  net.N = N;
  net.params = params;
  auto dal = [](void** p, size_t b) {
    if (cudaMalloc(p, b) != cudaSuccess) throw EfieError{-2, "precond: cudaMalloc failed"};
  };
  dal((void**)&net.P, sizeof(float) * NPARAM);
  dal((void**)&net.Wcat, sizeof(__nv_bfloat16) * NL * NW * 128);
  dal((void**)&net.WcatT, sizeof(__nv_bfloat16) * NL * NW * 128);
  dal((void**)&net.nbr, sizeof(int32_t) * 4 * N);
  dal((void**)&net.sgn, sizeof(float) * 4 * N);
  dal((void**)&net.lnorm, sizeof(float) * N);
  dal((void**)&net.red, sizeof(double) * 4);
  for (int l = 0; l <= NL; ++l) dal((void**)&net.h[l], sizeof(float) * N * NW);
  dal((void**)&net.x, sizeof(float) * N * NIN);
  cudaMemcpy(net.P, params.data(), sizeof(float) * NPARAM, cudaMemcpyHostToDevice);
  cudaMemcpy(net.nbr, nbr.data(), sizeof(int32_t) * 4 * N, cudaMemcpyHostToDevice);
  cudaMemcpy(net.sgn, sgn.data(), sizeof(float) * 4 * N, cudaMemcpyHostToDevice);
  cudaMemcpy(net.lnorm, lnorm.data(), sizeof(float) * N, cudaMemcpyHostToDevice);
  if (training) {
    dal((void**)&net.G, sizeof(float) * NPARAM);
    dal((void**)&net.M, sizeof(float) * NPARAM);
    dal((void**)&net.V, sizeof(float) * NPARAM);
    cudaMemset(net.M, 0, sizeof(float) * NPARAM);
    cudaMemset(net.V, 0, sizeof(float) * NPARAM);
    dal((void**)&net.u0, sizeof(float) * N * NW);
    for (int l = 0; l < NL; ++l) {
      dal((void**)&net.u[l], sizeof(float) * N * NW);
      dal((void**)&net.a[l], sizeof(float) * N * NW);
    }
    dal((void**)&net.dh, sizeof(float) * N * NW);
    dal((void**)&net.du, sizeof(float) * N * NW);
    dal((void**)&net.dXa, sizeof(float) * N * NW);
    dal((void**)&net.part, sizeof(float) * NB_RED * PART_W);
    dal((void**)&net.dpart, sizeof(double) * NB_RED * 2);
  }
  k_nn_pack<<<64, 256>>>(net.P, net.Wcat, net.WcatT);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) throw EfieError{-3, std::string("precond setup: ") + cudaGetErrorString(e)};
}

void nn_free(Net& net) {
  void* ps[] = {net.P, net.G, net.M, net.V, net.Wcat, net.WcatT, net.nbr, net.sgn, net.lnorm, net.x, net.u0,
                net.dh, net.du, net.dXa, net.red, net.part, net.dpart};
  for (void* p : ps)
    if (p) cudaFree(p);
  for (int l = 0; l <= NL; ++l)
    if (net.h[l]) cudaFree(net.h[l]);
  for (int l = 0; l < NL; ++l) {
    if (net.u[l]) cudaFree(net.u[l]);
    if (net.a[l]) cudaFree(net.a[l]);
  }
  net = Net();
}

// z = net(r) for one vector (canonical order), c128 in and out.
void nn_forward(Net& net, const double2* r, double2* z, bool training, cudaStream_t s) {
  const int64_t N = net.N;
  launch_norms(r, N, N, 1, net.red, s);
  k_nn_encode<<<(unsigned)grid_for(N * NW, 256), 256, 0, s>>>(r, net.lnorm, N, net.red, net.P,
                                                             training ? net.x : nullptr,
                                                             training ? net.u0 : nullptr, net.h[0]);
  const unsigned tiles = (unsigned)((N + TILE - 1) / TILE);
  for (int l = 0; l < NL; ++l)
    k_nn_layer<<<tiles, 128, 0, s>>>(net.h[l], net.nbr, net.sgn, N, net.Wcat + l * NW * 128,
                                     net.P + OFF_L0 + l * LAYER_SZ + 2 * NW * NW, net.h[l + 1],
                                     training ? net.u[l] : nullptr, training ? net.a[l] : nullptr);
  k_nn_decode<<<(unsigned)grid_for(N * 32, 256), 256, 0, s>>>(net.h[NL], N, net.P, net.red, z);
}

// Backward from g = dL/dz (forward must have run with training = true on the
// same input); parameter gradients are accumulated into G.
void nn_backward_g(Net& net, const double2* gz, cudaStream_t s) {
  const int64_t N = net.N;
  // fixed block counts (functions of N only) keep the summation order fixed
  const int nb_el = (int)std::min<int64_t>(NB_RED, (N * NW + 255) / 256);
  const int64_t tiles = (N + TILE - 1) / TILE;
  const int nb_tile = (int)std::min<int64_t>(NB_RED, tiles);
  k_nn_decode_back<<<nb_el, 256, 0, s>>>(net.h[NL], gz, N, net.red, net.P, net.part, net.dh);
  k_nn_reduce<<<(2 * NW + 2 + 127) / 128, 128, 0, s>>>(net.part, nb_el, 2 * NW + 2, net.G + OFF_WD);
  for (int l = NL - 1; l >= 0; --l) {
    k_nn_du<<<(unsigned)grid_for(N * NW, 256), 256, 0, s>>>(net.dh, net.u[l], net.du, N * NW);
    // dh stays as the residual-path gradient and receives dX_h and the neighbour part
    const size_t smem = sizeof(__nv_bfloat16) * (NW * (TILE + 8) + 128 * (TILE + 8) + TILE * (NW + 8) + 128 * (NW + 8));
    static SmemAttr attr;
    smem_attr_once(k_nn_layer_back, (int)smem, attr.v);
    k_nn_layer_back<<<nb_tile, 128, smem, s>>>(net.du, net.h[l], net.a[l], N, net.WcatT + l * NW * 128, net.part,
                                               net.dh, net.dXa);
    k_nn_reduce<<<(PART_W + 127) / 128, 128, 0, s>>>(net.part, nb_tile, PART_W, net.G + OFF_L0 + l * LAYER_SZ);
    k_nn_gather_back<<<(unsigned)grid_for(N * NW, 256), 256, 0, s>>>(net.dXa, net.nbr, net.sgn, N, net.dh);
  }
  k_nn_du<<<(unsigned)grid_for(N * NW, 256), 256, 0, s>>>(net.dh, net.u0, net.du, N * NW);
  k_nn_encode_back<<<nb_el, 256, 0, s>>>(net.du, net.x, N, net.part);
  k_nn_reduce<<<(NW * (NIN + 1) + 127) / 128, 128, 0, s>>>(net.part, nb_el, NW * (NIN + 1), net.G + OFF_WE);
}

// error loss |z - e|^2 / |e|^2: loss terms in red[1..2], gradient into G
// (gbuf: N complex scratch)
void nn_backward(Net& net, const double2* z, const double2* e, double2* gbuf, cudaStream_t s) {
  const int64_t N = net.N;
  const int nb = (int)std::min<int64_t>(NB_RED, (N + 255) / 256);
  k_nn_loss<<<nb, 256, 0, s>>>(z, e, N, net.dpart);
  k_nn_loss_reduce<<<1, 32, 0, s>>>(net.dpart, nb, net.red + 1);
  k_nn_err_grad<<<(unsigned)grid_for(N, 256), 256, 0, s>>>(z, e, N, net.red + 1, gbuf);
  nn_backward_g(net, gbuf, s);
}

void nn_zero_grad(Net& net, cudaStream_t s) { cudaMemsetAsync(net.G, 0, sizeof(float) * NPARAM, s); }

void nn_adam(Net& net, float lr, float gscale, cudaStream_t s) {
  net.step++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)net.step), c2 = 1.f - powf(b2, (float)net.step);
  k_adam<<<64, 256, 0, s>>>(net.P, net.G, net.M, net.V, NPARAM, lr, b1, b2, 1e-8f, c1, c2, gscale);
  k_nn_pack<<<64, 256, 0, s>>>(net.P, net.Wcat, net.WcatT);
}

void nn_read_params(Net& net, std::vector<float>& out) {
  out.resize(NPARAM);
  cudaMemcpy(out.data(), net.P, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost);
}
void nn_read_grads(Net& net, std::vector<float>& out) {
  out.resize(NPARAM);
  cudaMemcpy(out.data(), net.G, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost);
}
void nn_loss_terms(Net& net, double* num, double* den) {
  double t[2];
  cudaMemcpy(t, net.red + 1, sizeof(double) * 2, cudaMemcpyDeviceToHost);
  *num = t[0];
  *den = t[1];
}

}  // namespace efie
