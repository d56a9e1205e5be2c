// Top-grid-level translation on the 5th-generation tensor cores (tcgen05).
//
// On the top grid level every box translates every non-adjacent box (Sec. IV,
// the last level that carries grids), so for one frequency f the translation
//   R^[f][x][c] = sum_y K^[f][o(x - y)] Q^[f][y][c]
// is a dense complex matrix product: targets x sources (the kernel spectrum
// gathered through the box-offset index, zero for adjacent pairs) times
// sources x channels (the source spectra).  One CTA computes one target tile
// (<= 128 targets, one TMEM lane each) of one frequency for 32 channels.
//
// Precision: the far field is complex FP32.  The tensor cores take TF32
// operands (10 explicit mantissa bits), so every FP32 operand is split as
// x = x_hi + x_lo with x_hi = tf32(x), x_lo = tf32(x - x_hi), and each real
// product is a_hi b_hi + a_hi b_lo + a_lo b_hi (the a_lo b_lo term is below
// FP32 rounding), accumulated in FP32 in TMEM: FP32-class products at the
// tensor-core rate.  The complex product takes four real ones:
//   D_r = K_r Q_r - K_i Q_i,  D_i = K_r Q_i + K_i Q_r.
//
// Data flow per CTA: the kernel spectrum row of f (O complex values) is staged
// in shared memory once; sources go in chunks of KC = 16; for each chunk every
// thread gathers the kernel values of its target row through the index tile,
// splits them and writes the four A operands (K_r hi/lo, K_i hi/lo; 16 TMEM
// columns each) into TMEM with tcgen05.st, and the CTA writes the four B
// operands (Q_r hi/lo, Q_i hi/lo; 16 sources x 32 channels) into shared
// memory in the canonical K-major core-matrix layout.  One thread issues the
// 24 MMAs of the chunk (2 k-steps of 8 x 12 split products) and commits them
// to the chunk buffer's mbarrier.  Two buffers: the next chunk is built while
// the tensor cores run the current one.  The accumulators D_r, D_i (32 FP32
// columns each) are read back with tcgen05.ld and stored as complex rows.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "device_api.cuh"

namespace efie {

namespace {

constexpr int TC_KC = 16;                  // sources per chunk
constexpr int TC_C = 32;                   // channels (8 right-hand sides x 4 components)
constexpr int TC_LBO = 128;                // bytes between core matrices along K (sources)
constexpr int TC_SBO = (TC_KC / 4) * 128;  // bytes between core matrices along N (channels)
constexpr int TC_BVAR = TC_C * TC_KC * 4;  // bytes of one B operand (2 KB)
constexpr int TC_BBUF = 4 * TC_BVAR;       // one chunk buffer: Q_r hi/lo, Q_i hi/lo
constexpr uint32_t TC_COLS = 256;          // TMEM columns per CTA (2 CTAs per SM)
constexpr uint32_t TC_ACOL = 64;           // A buffers start here; D_r at 0, D_i at 32
constexpr long long TC_SPIN = 1LL << 20;   // iteration limit of every mbarrier wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// tf32 rounding (round to nearest, ties away) of an FP32 value, kept in FP32
__device__ __forceinline__ float tf32r(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// shared-memory matrix descriptor: K-major, no swizzle, 8 x 16-byte core matrices
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((TC_LBO >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((TC_SBO >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of this architecture
  return d;
}

// instruction descriptor: kind::tf32, FP32 accumulate, A and B K-major,
// M = 128, N = 32; bit 13 negates A
__host__ __device__ constexpr uint32_t tc_idesc(bool negA) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (negA ? (1u << 13) : 0u) | ((uint32_t)(TC_C >> 3) << 17) |
         ((128u >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n" ::"r"(
          taddr),
      "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "f"(v[8]), "f"(v[9]),
      "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15]));
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%"
      "19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]), "=f"(v[8]),
        "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]), "=f"(v[15]), "=f"(v[16]),
        "=f"(v[17]), "=f"(v[18]), "=f"(v[19]), "=f"(v[20]), "=f"(v[21]), "=f"(v[22]), "=f"(v[23]), "=f"(v[24]),
        "=f"(v[25]), "=f"(v[26]), "=f"(v[27]), "=f"(v[28]), "=f"(v[29]), "=f"(v[30]), "=f"(v[31])
      : "r"(taddr));
}

// bounded wait for the completion of phase `parity` of an mbarrier; false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (long long it = 0; it < TC_SPIN; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void cp16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem));
}
__device__ __forceinline__ void cp8(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(smem)), "l"(gmem));
}

}  // namespace

// grid: (tile, frequency); 128 threads; dynamic shared memory:
//   [0, kbytes)               kernel spectrum row of the frequency (O complex)
//   [kbytes, + 2 TC_BBUF)     B operands of the two chunk buffers
// `err` (host-mapped) is set to 1 if an mbarrier wait runs out; the tile's
// outputs are then NaN.
__global__ void __launch_bounds__(128, 2)
    k_mac_top_tc(const float2* __restrict__ Qh, float2* __restrict__ Rh, const float2* __restrict__ Kh, int64_t B,
                 int64_t O, int64_t nf, const int64_t* __restrict__ tgt_ptr, const int32_t* __restrict__ tgt,
                 const int64_t* __restrict__ src_ptr, const int32_t* __restrict__ src,
                 const int64_t* __restrict__ kidx_off, const int32_t* __restrict__ kidx, int64_t f0,
                 int kbytes, int* err) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t mbar[2];
  float2* Ks = reinterpret_cast<float2*>(tc_smem);
  unsigned char* Bs = tc_smem + kbytes;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int tile = blockIdx.x;
  const int64_t f = f0 + blockIdx.y;
  if (f >= nf) return;
  const int64_t t0 = tgt_ptr[tile], nt = tgt_ptr[tile + 1] - t0;
  const int64_t s0 = src_ptr[tile], ns = src_ptr[tile + 1] - s0;
  const int tpad = (int)(((nt + 7) / 8) * 8);
  const int32_t* kb = kidx + kidx_off[tile];
  const float2* Qf = Qh + f * B * TC_C;
  // an earlier CTA's wait ran out: skip the work (outputs NaN), take no TMEM
  if (err && *reinterpret_cast<volatile int*>(err)) {
    const float v = __int_as_float(0x7fc00000);
    if (tid < nt)
      for (int n = 0; n < TC_C; n += 2)
        *reinterpret_cast<float4*>(Rh + f * B * TC_C + (int64_t)tgt[t0 + tid] * TC_C + n) = make_float4(v, v, v, v);
    return;
  }

  // stage the kernel spectrum row of f (16-byte copies when the row is aligned)
  {
    const float2* Kf = Kh + f * O;
    if ((((uintptr_t)Kf) & 15) == 0) {
      const int64_t n16 = O / 2;
      for (int64_t i = tid; i < n16; i += 128) cp16(Ks + 2 * i, Kf + 2 * i);
      if ((O & 1) && tid == 0) cp8(Ks + O - 1, Kf + O - 1);
    } else {
      for (int64_t i = tid; i < O; i += 128) cp8(Ks + i, Kf + i);
    }
    asm volatile("cp.async.commit_group;\n" ::);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                 "r"(TC_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;\n");
  }
  asm volatile("cp.async.wait_all;\n" ::);
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tm = tmem_base;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const int nchunks = (int)((ns + TC_KC - 1) / TC_KC);
  bool ok = true;

  // index tile rows of a chunk for this thread's target (prefetched one chunk ahead)
  int32_t idn[TC_KC];
  auto load_idx = [&](int c) {
#pragma unroll
    for (int j = 0; j < TC_KC; ++j) {
      const int64_t jj = (int64_t)c * TC_KC + j;
      idn[j] = (c < nchunks && jj < ns && tid < tpad) ? __ldg(kb + jj * tpad + tid) : -1;
    }
  };
  // source spectra of a chunk (4 complex values per thread, prefetched)
  float2 qn[4];
  auto load_q = [&](int c) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + 128 * u, j = e >> 5, n = e & 31;
      const int64_t jj = (int64_t)c * TC_KC + j;
      qn[u] = make_float2(0.f, 0.f);
      if (c < nchunks && jj < ns) {
        const int32_t y = __ldg(src + s0 + jj);
        qn[u] = __ldg(Qf + (int64_t)y * TC_C + n);
      }
    }
  };
  load_idx(0);
  load_q(0);

  for (int c = 0; c < nchunks; ++c) {
    const int b = c & 1;
    // buffer b was last used by chunk c - 2: wait for its MMAs
    if (c >= 2) ok = ok && mbar_wait(smem_u32(&mbar[b]), (uint32_t)(((c - 2) >> 1) & 1));
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    int32_t idc[TC_KC];
#pragma unroll
    for (int j = 0; j < TC_KC; ++j) idc[j] = idn[j];
    float2 qc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) qc[u] = qn[u];
    load_idx(c + 1);
    load_q(c + 1);
    // A operands of this thread's target row -> TMEM columns of buffer b
    {
      float arh[TC_KC], arl[TC_KC], aih[TC_KC], ail[TC_KC];
#pragma unroll
      for (int j = 0; j < TC_KC; ++j) {
        const float2 kv = idc[j] >= 0 ? Ks[idc[j]] : make_float2(0.f, 0.f);
        arh[j] = tf32r(kv.x);
        arl[j] = tf32r(kv.x - arh[j]);
        aih[j] = tf32r(kv.y);
        ail[j] = tf32r(kv.y - aih[j]);
      }
      const uint32_t ta = tm + lane_base + TC_ACOL + (uint32_t)b * 4 * TC_KC;
      tmem_st16(ta + 0 * TC_KC, arh);
      tmem_st16(ta + 1 * TC_KC, arl);
      tmem_st16(ta + 2 * TC_KC, aih);
      tmem_st16(ta + 3 * TC_KC, ail);
    }
    // B operands -> shared memory (K-major core matrices: (n, k) at
    // (n/8) SBO + (k/4) LBO + (n%8) 16 + (k%4) 4 bytes)
    {
      unsigned char* bb = Bs + b * TC_BBUF;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = tid + 128 * u, j = e >> 5, n = e & 31;
        const int off = (n >> 3) * TC_SBO + (j >> 2) * TC_LBO + (n & 7) * 16 + (j & 3) * 4;
        const float rh = tf32r(qc[u].x), ih = tf32r(qc[u].y);
        *reinterpret_cast<float*>(bb + 0 * TC_BVAR + off) = rh;
        *reinterpret_cast<float*>(bb + 1 * TC_BVAR + off) = tf32r(qc[u].x - rh);
        *reinterpret_cast<float*>(bb + 2 * TC_BVAR + off) = ih;
        *reinterpret_cast<float*>(bb + 3 * TC_BVAR + off) = tf32r(qc[u].y - ih);
      }
    }
    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t dr = tm, di = tm + TC_C;
      const uint32_t a0 = tm + TC_ACOL + (uint32_t)b * 4 * TC_KC;
      const uint32_t bs = smem_u32(Bs + b * TC_BBUF);
#pragma unroll
      for (int kk = 0; kk < TC_KC / 8; ++kk) {
        const uint32_t arh = a0 + 0 * TC_KC + kk * 8, arl = a0 + 1 * TC_KC + kk * 8;
        const uint32_t aih = a0 + 2 * TC_KC + kk * 8, ail = a0 + 3 * TC_KC + kk * 8;
        const uint32_t ko = (uint32_t)kk * 2 * TC_LBO;
        const uint64_t brh = smem_desc(bs + 0 * TC_BVAR + ko), brl = smem_desc(bs + 1 * TC_BVAR + ko);
        const uint64_t bih = smem_desc(bs + 2 * TC_BVAR + ko), bil = smem_desc(bs + 3 * TC_BVAR + ko);
        const uint32_t acc0 = (c > 0 || kk > 0) ? 1u : 0u;
        const uint32_t ip = tc_idesc(false), in = tc_idesc(true);
        // D_r = K_r Q_r - K_i Q_i
        mma_tf32(dr, arh, brh, ip, acc0);
        mma_tf32(dr, arh, brl, ip, 1u);
        mma_tf32(dr, arl, brh, ip, 1u);
        mma_tf32(dr, aih, bih, in, 1u);
        mma_tf32(dr, aih, bil, in, 1u);
        mma_tf32(dr, ail, bih, in, 1u);
        // D_i = K_r Q_i + K_i Q_r
        mma_tf32(di, arh, bih, ip, acc0);
        mma_tf32(di, arh, bil, ip, 1u);
        mma_tf32(di, arl, bih, ip, 1u);
        mma_tf32(di, aih, brh, ip, 1u);
        mma_tf32(di, aih, brl, ip, 1u);
        mma_tf32(di, ail, brh, ip, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       smem_u32(&mbar[b]))
                   : "memory");
    }
  }
  // all MMAs done: the last commit covers every earlier one of the issuing thread
  if (nchunks > 0) ok = mbar_wait(smem_u32(&mbar[(nchunks - 1) & 1]), (uint32_t)(((nchunks - 1) >> 1) & 1)) && ok;
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (!ok && err) *reinterpret_cast<volatile int*>(err) = 1;
  if (tid < nt) {
    float2* out = Rh + f * B * TC_C + (int64_t)tgt[t0 + tid] * TC_C;
    if (nchunks == 0 || !ok) {
      const float v = ok ? 0.f : __int_as_float(0x7fc00000);
      for (int n = 0; n < TC_C; n += 2) *reinterpret_cast<float4*>(out + n) = make_float4(v, v, v, v);
    }
  }
  if (nchunks > 0 && ok) {
    float vr[TC_C], vi[TC_C];
    tmem_ld32(tm + lane_base, vr);
    tmem_ld32(tm + lane_base + TC_C, vi);
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
    if (tid < nt) {
      float2* out = Rh + f * B * TC_C + (int64_t)tgt[t0 + tid] * TC_C;
#pragma unroll
      for (int n = 0; n < TC_C; n += 2)
        *reinterpret_cast<float4*>(out + n) = make_float4(vr[n], vi[n], vr[n + 1], vi[n + 1]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tm), "r"(TC_COLS));
}

// Returns false when the configuration does not fit this kernel (the caller
// then uses the CUDA-core kernels): 32 channels, tiles of 9..128 targets, and
// a kernel spectrum row that fits in shared memory beside the B buffers with
// two CTAs per SM.
static int64_t tc_smem_bytes(int64_t O) {
  const int64_t kbytes = ((O * 8 + 1023) / 1024) * 1024;
  // at least 80 KB per CTA, so that no more than two CTAs (2 x 256 TMEM
  // columns) are resident on an SM and a TMEM allocation never waits
  return std::max<int64_t>(kbytes + 2 * TC_BBUF, 80 * 1024);
}

bool mac_top_tc_fits(int C, int max_tile_targets, int64_t O) {
  return C == TC_C && max_tile_targets > 8 && max_tile_targets <= 128 && O > 0 && tc_smem_bytes(O) <= 110 * 1024;
}

bool launch_mac_top_tc(const float2* Qh, float2* Rh, const float2* Kh, int64_t B, int C, int64_t O, int64_t nf,
                       int64_t ntiles, int max_tile_targets, const int64_t* tgt_ptr, const int32_t* tgt,
                       const int64_t* src_ptr, const int32_t* src, const int64_t* kidx_off, const int32_t* kidx,
                       int* err, cudaStream_t s) {
  if (!mac_top_tc_fits(C, max_tile_targets, O)) return false;
  const int64_t kbytes = ((O * 8 + 1023) / 1024) * 1024;
  const int64_t smem = tc_smem_bytes(O);
  static std::atomic<uint64_t> attr{0};
  smem_attr_once(k_mac_top_tc, (int)smem, attr);
  for (int64_t fs = 0; fs < nf; fs += 65535) {
    const int64_t nfc = nf - fs < 65535 ? nf - fs : 65535;
    dim3 grid((unsigned)ntiles, (unsigned)nfc);
    k_mac_top_tc<<<grid, 128, (size_t)smem, s>>>(Qh, Rh, Kh, B, O, nf, tgt_ptr, tgt, src_ptr, src, kidx_off, kidx,
                                                 fs, (int)kbytes, err);
  }
  return true;
}

}  // namespace efie
