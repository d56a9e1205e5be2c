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

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float* v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};\n" ::"r"(taddr), "f"(v[0]),
               "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]));
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

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]), "=f"(v[8]),
        "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]), "=f"(v[15])
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

// ---------------------------------------------------------------------------
// Persistent, warp-specialised form (one CTA per SM, all 512 TMEM columns).
// The CTA owns frequencies f = blockIdx.x + k * gridDim.x and runs every tile
// of each; the chunks of 16 sources of all tiles form one sequence g.  Roles:
//   producers (2 warpgroups; chunk g goes to warpgroup g % 2): gather and
//     split the kernel values of their target row into the A stage of chunk g
//     (TMEM, tcgen05.st) and the source spectra into its B stage (shared
//     memory), then arrive on full[g % STG]; their global loads run ahead
//     (offset ids two chunks, spectra one chunk);
//   MMA warp (one lane): loads the kernel spectrum row of the next frequency
//     by TMA bulk copies while the current one is in use, waits on full[],
//     issues the 12 MMAs of a chunk (N = 64 NCH: B = [Q_r | Q_i] rows; the
//     hi x hi, hi x lo and lo x hi products of K_r into D1 and of K_i into
//     D2) and commits them to empty[g % STG], and after a tile's last chunk
//     to dfull[];
//   epilogue warpgroup: reads the tile's accumulators, forms
//     R_r = (K_r Q_r) - (K_i Q_i), R_i = (K_r Q_i) + (K_i Q_r), frees the
//     buffer (dempty[]) and stores the complex rows.
// One 8-RHS chunk per pass (NCH = 1): four chunk stages, two accumulator
// buffers; two chunks (NCH = 2): three stages, one accumulator buffer of 256
// columns.  Two kernel-row buffers; every mbarrier wait is bounded and a
// timeout stops every role of the CTA.
namespace {
constexpr int T2_PROD = 256;                  // producer threads (2 warpgroups)
constexpr int T2_MMA_WARP = T2_PROD / 32;     // warp 8
constexpr int T2_EPI0 = T2_PROD + 32;         // first epilogue thread
constexpr int T2_THREADS = T2_EPI0 + 128;     // 416 threads per CTA
constexpr uint32_t T2_COLS = 512;
constexpr uint32_t T2_A0 = 256;               // A stages at 256 + 64 * stage
constexpr int T2_PIECE = 16384;               // bytes per bulk copy of a kernel row
// Per NCH (8-right-hand-side chunks per pass: 1 or 2):
//   B rows: 32 NCH channels real, then 32 NCH imaginary (N = 64 NCH)
//   accumulator buffer: D1 = K_r B (64 NCH columns) | D2 = K_i B; two buffers
//   for NCH = 1, one for NCH = 2 (256 columns)
//   chunk stages: 4 for NCH = 1, 3 for NCH = 2 (shared memory)
template <int NCH>
struct T2Cfg {
  static constexpr int BN = 64 * NCH;
  static constexpr int BMAT = BN * TC_KC * 4;
  static constexpr int BSTAGE = 2 * BMAT;
  static constexpr int STG = NCH == 1 ? 4 : 3;
  static constexpr int DB = NCH == 1 ? 2 : 1;
  static constexpr uint32_t DBUF = 128u * NCH;
  static constexpr uint32_t IDESC =
      (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) | ((128u >> 4) << 24);
};
constexpr int T2_STAGES = 4;                  // largest stage count (barrier arrays)

struct T2Tile {
  int64_t koff;        // start of the tile's index block
  int64_t s0;          // start of the tile's source list
  int32_t t0, nt, tpad, ns;
};
struct T2Bar {
  uint64_t full[T2_STAGES], empty[T2_STAGES], dfull[2], dempty[2], rfull[2], rempty[2];
  uint32_t tmem_base;
  int abort;
  int nq;
};

// x = hi + lo with hi the TF32 part of x (sign, exponent and 10 mantissa bits
// kept, the rest cleared) and lo = x - hi exactly; the tensor core truncates lo
// to TF32 in turn, so x is carried to about 22 bits
__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

__device__ __forceinline__ void mbar_init(uint64_t* b, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(b)) : "memory");
}
// bounded wait that also gives up at once when another role of the CTA gave
// up (abort, a shared-memory flag of the CTA)
__device__ __forceinline__ bool t2_wait(uint64_t* b, uint32_t parity, int* abort, int* err) {
  const uint32_t a = smem_u32(b);
  for (long long it = 0; it < TC_SPIN; ++it) {
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
__device__ __forceinline__ bool t2_wait(uint64_t* b, uint32_t parity, T2Bar* bar, int* err) {
  return t2_wait(b, parity, &bar->abort, err);
}

__device__ __forceinline__ uint64_t smem_desc_sbo(uint32_t saddr, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((TC_LBO >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
}  // namespace

// dynamic shared memory: [2 kernel rows of kbytes][STG B stages][tile table
// (ntiles T2Tile)][chunk table (nq_cap entries)].  Chunk c < NCH of the pass
// has its spectra at Qh[c] and writes Rh[c]; source j of tile t is box
// src[src_ptr[t] + j].
template <int NCH>
__global__ void __maxnreg__(128)
    k_mac_top_tc2(const float2* __restrict__ Qh0, const float2* __restrict__ Qh1, float2* __restrict__ Rh0,
                  float2* __restrict__ Rh1, const float2* __restrict__ Kh, int64_t B,
                  int64_t O, int64_t nf, int64_t ntiles, const int64_t* __restrict__ tgt_ptr,
                  const int32_t* __restrict__ tgt, const int64_t* __restrict__ src_ptr,
                  const int32_t* __restrict__ src, const int64_t* __restrict__ kidx_off,
                  const int16_t* __restrict__ kidx, int kbytes, int nq_cap, int* err) {
  extern __shared__ __align__(1024) unsigned char t2_smem[];
  __shared__ T2Bar bar;
  unsigned char* rows = t2_smem;
  unsigned char* Bs = t2_smem + 2 * kbytes;
  using Cfg = T2Cfg<NCH>;
  T2Tile* tiles = reinterpret_cast<T2Tile*>(Bs + Cfg::STG * Cfg::BSTAGE);
  uint32_t* ctab = reinterpret_cast<uint32_t*>(tiles + ntiles);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t K = nf > blockIdx.x ? (nf - 1 - blockIdx.x) / gridDim.x + 1 : 0;   // frequencies of this CTA

  if (tid == 0) {
    for (int i = 0; i < Cfg::STG; ++i) {
      mbar_init(&bar.full[i], 128);
      mbar_init(&bar.empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bar.dfull[i], 1);
      mbar_init(&bar.dempty[i], 128);
      mbar_init(&bar.rfull[i], 1);
      mbar_init(&bar.rempty[i], T2_PROD);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    bar.abort = 0;
    // tile table and chunk table ((tile << 16) | first source, tile by tile)
    int q = 0;
    for (int64_t t = 0; t < ntiles; ++t) {
      const int64_t ns = src_ptr[t + 1] - src_ptr[t], nt = tgt_ptr[t + 1] - tgt_ptr[t];
      tiles[t].koff = kidx_off[t];
      tiles[t].s0 = src_ptr[t];
      tiles[t].t0 = (int32_t)tgt_ptr[t];
      tiles[t].nt = (int32_t)nt;
      tiles[t].tpad = (int32_t)(((nt + 7) / 8) * 8);
      tiles[t].ns = (int32_t)ns;
      for (int64_t j0 = 0; j0 < ns && q < nq_cap; j0 += TC_KC) ctab[q++] = (uint32_t)((t << 16) | j0);
    }
    bar.nq = q;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&bar.tmem_base)),
                 "r"(T2_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tm = bar.tmem_base;
  const int64_t nq = bar.nq;
  const int64_t TS = K * ntiles;      // tiles of this CTA

  if (tid < T2_PROD) {
    // ------------------------------------------------------------ producers
    const int wg = tid >> 7, r = tid & 127;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    // B operands: this thread stores source jB of the chunk, channels chB + 8u
    // of pass chunk u / 4: row u * 8 + chB (real) and 32 NCH + u * 8 + chB
    // (imaginary), i.e. core group u and 4 NCH + u
    const int jB = (warp & 3) * 4 + (lane >> 3), chB = lane & 7;
    const int boff = (jB >> 2) * TC_LBO + (jB & 3) * 4 + chB * 16;
    const int nq32 = (int)nq;
    float2 qn[4 * NCH];
    // Loads run ahead of use: the index words of a chunk two chunks ahead,
    // the source box of this thread's B row one chunk ahead of the spectra
    // that depend on it, the spectra one chunk ahead.
    // index words of chunk (k, q): its 16 sources of target row r, int16,
    // packed two per word (the block [chunk][tpad][16] of the tile)
    auto load_k = [&](int64_t k, int q, uint32_t (&w)[TC_KC / 2]) {
#pragma unroll
      for (int i = 0; i < TC_KC / 2; ++i) w[i] = 0xFFFFFFFFu;
      if (k >= K) return;
      const uint32_t e = ctab[q];
      const T2Tile& T = tiles[e >> 16];
      const int j0 = (int)(e & 0xFFFFu);
      if (r < T.tpad) {
        const uint4* kb = reinterpret_cast<const uint4*>(kidx + T.koff + ((int64_t)(j0 / TC_KC) * T.tpad + r) * TC_KC);
        const uint4 a = __ldg(kb), b = __ldg(kb + 1);
        w[0] = a.x, w[1] = a.y, w[2] = a.z, w[3] = a.w, w[4] = b.x, w[5] = b.y, w[6] = b.z, w[7] = b.w;
      }
    };
    // source box of this thread's B row in chunk (k, q), or -1
    auto load_src = [&](int64_t k, int q) -> int32_t {
      if (k >= K) return -1;
      const uint32_t e = ctab[q];
      const T2Tile& T = tiles[e >> 16];
      const int j0 = (int)(e & 0xFFFFu);
      return j0 + jB < T.ns ? __ldg(src + T.s0 + j0 + jB) : -1;
    };
    auto load_q = [&](int64_t k, int32_t y) {
#pragma unroll
      for (int u = 0; u < 4 * NCH; ++u) qn[u] = make_float2(0.f, 0.f);
      if (k >= K || y < 0) return;
      const int64_t o = ((int64_t)(blockIdx.x + k * gridDim.x) * B + y) * TC_C + chB;
#pragma unroll
      for (int u = 0; u < 4; ++u) qn[u] = __ldg(Qh0 + o + 8 * u);
      if (NCH == 2) {
#pragma unroll
        for (int u = 0; u < 4; ++u) qn[4 + u] = __ldg(Qh1 + o + 8 * u);
      }
    };
    // this warpgroup's chunks g = wg, wg + 2, ... as (frequency k, chunk q):
    // (kn, qn_) the next one, (kn2, qn2) the one after it
    auto advance = [&](int64_t& kk, int& qq) {
      qq += 2;
      while (qq >= nq32) {
        qq -= nq32;
        ++kk;
      }
    };
    int64_t kn = 0;
    int qn_ = wg;
    while (qn_ >= nq32 && nq32 > 0) {
      qn_ -= nq32;
      ++kn;
    }
    int64_t kn2 = kn;
    int qn2 = qn_;
    uint32_t kwA[TC_KC / 2], kwB[TC_KC / 2];
    int32_t yB = -1;
#pragma unroll
    for (int i = 0; i < TC_KC / 2; ++i) kwA[i] = kwB[i] = 0xFFFFFFFFu;
    if (nq32 > 0) {
      load_k(kn, qn_, kwA);
      load_q(kn, load_src(kn, qn_));
      advance(kn2, qn2);
      load_k(kn2, qn2, kwB);
      yB = load_src(kn2, qn2);
    }
    int64_t g = wg;
    bool ok = true;
    for (int64_t k = 0; k < K && ok; ++k) {
      const int rb = (int)(k & 1);
      ok = t2_wait(&bar.rfull[rb], (uint32_t)((k >> 1) & 1), &bar, err);
      if (!ok) break;
      const float2* Ks = reinterpret_cast<const float2*>(rows + rb * kbytes);
      for (; g < (k + 1) * nq; g += 2) {
        int32_t idc[TC_KC];
        float2 qc[4 * NCH];
#pragma unroll
        for (int j = 0; j < TC_KC; ++j) idc[j] = (int32_t)(int16_t)(kwA[j >> 1] >> ((j & 1) * 16));
#pragma unroll
        for (int u = 0; u < 4 * NCH; ++u) qc[u] = qn[u];
        // chunk after this one: index words already here, spectra now; the
        // one after that: index words and source box now
#pragma unroll
        for (int i = 0; i < TC_KC / 2; ++i) kwA[i] = kwB[i];
        load_q(kn2, yB);
        advance(kn2, qn2);
        load_k(kn2, qn2, kwB);
        yB = load_src(kn2, qn2);
        const uint32_t gu = (uint32_t)g;
        const int slot = (int)(gu % Cfg::STG);
        if (gu >= (uint32_t)Cfg::STG) {
          ok = t2_wait(&bar.empty[slot], ((gu / Cfg::STG) - 1) & 1, &bar, err);
          if (!ok) break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        {
          const uint32_t ta = tm + lane_base + T2_A0 + (uint32_t)slot * 4 * TC_KC;
#pragma unroll
          for (int hh = 0; hh < TC_KC; hh += 8) {
            float arh[8], arl[8], aih[8], ail[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const float2 kv = idc[hh + j] >= 0 ? Ks[idc[hh + j]] : make_float2(0.f, 0.f);
              arh[j] = tf32_hi(kv.x);
              arl[j] = kv.x - arh[j];
              aih[j] = tf32_hi(kv.y);
              ail[j] = kv.y - aih[j];
            }
            tmem_st8(ta + 0 * TC_KC + hh, arh);
            tmem_st8(ta + 1 * TC_KC + hh, arl);
            tmem_st8(ta + 2 * TC_KC + hh, aih);
            tmem_st8(ta + 3 * TC_KC + hh, ail);
          }
        }
        {
          float* bb = reinterpret_cast<float*>(Bs + slot * Cfg::BSTAGE + boff);
#pragma unroll
          for (int u = 0; u < 4 * NCH; ++u) {
            const float rh = tf32_hi(qc[u].x), ih = tf32_hi(qc[u].y);
            bb[(u * TC_SBO) / 4] = rh;
            bb[((4 * NCH + u) * TC_SBO) / 4] = ih;
            bb[(Cfg::BMAT + u * TC_SBO) / 4] = qc[u].x - rh;
            bb[(Cfg::BMAT + (4 * NCH + u) * TC_SBO) / 4] = qc[u].y - ih;
          }
        }
        asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        mbar_arrive(&bar.full[slot]);
      }
      if (!ok) break;
      mbar_arrive(&bar.rempty[rb]);   // this thread is done with the row buffer
    }
  } else if (warp == T2_MMA_WARP) {
    // ------------------------------------------------------------ MMA warp
    if (lane == 0) {
      auto load_row = [&](int64_t k) {
        const int rb = (int)(k & 1);
        const unsigned char* src = reinterpret_cast<const unsigned char*>(Kh + (blockIdx.x + k * gridDim.x) * O);
        const uint32_t dst = smem_u32(rows + rb * kbytes);
        const uint32_t bytes = (uint32_t)(O * 8);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(&bar.rfull[rb])),
                     "r"(bytes)
                     : "memory");
        for (uint32_t off = 0; off < bytes; off += T2_PIECE) {
          const uint32_t n = bytes - off < (uint32_t)T2_PIECE ? bytes - off : (uint32_t)T2_PIECE;
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst +
                                                                                                                  off),
              "l"(src + off), "r"(n), "r"(smem_u32(&bar.rfull[rb]))
              : "memory");
        }
      };
      bool ok = true;
      if (K > 0) load_row(0);
      if (K > 1) load_row(1);
      int64_t g = 0, ts = 0;
      for (int64_t k = 0; k < K && ok; ++k) {
        if (k >= 1 && k + 1 < K) {
          ok = t2_wait(&bar.rempty[(k + 1) & 1], (uint32_t)(((k - 1) >> 1) & 1), &bar, err);
          if (!ok) break;
          load_row(k + 1);
        }
        for (int64_t t = 0; t < ntiles && ok; ++t, ++ts) {
          const uint32_t tsu = (uint32_t)ts;
          const int db = (int)(tsu % Cfg::DB);
          if (tsu >= (uint32_t)Cfg::DB) {
            ok = t2_wait(&bar.dempty[db], ((tsu / Cfg::DB) - 1) & 1, &bar, err);
            if (!ok) break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
          const int64_t nch = (tiles[t].ns + TC_KC - 1) / TC_KC;
          const uint32_t d1 = tm + (uint32_t)db * Cfg::DBUF, d2 = d1 + 64 * NCH;
          for (int64_t c = 0; c < nch; ++c, ++g) {
            const uint32_t gu = (uint32_t)g;
            const int slot = (int)(gu % Cfg::STG);
            ok = t2_wait(&bar.full[slot], (gu / Cfg::STG) & 1, &bar, err);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t a0 = tm + T2_A0 + (uint32_t)slot * 4 * TC_KC;
            const uint32_t bs = smem_u32(Bs + slot * Cfg::BSTAGE);
#pragma unroll
            for (int kk = 0; kk < TC_KC / 8; ++kk) {
              const uint32_t arh = a0 + 0 * TC_KC + kk * 8, arl = a0 + 1 * TC_KC + kk * 8;
              const uint32_t aih = a0 + 2 * TC_KC + kk * 8, ail = a0 + 3 * TC_KC + kk * 8;
              const uint32_t ko = (uint32_t)kk * 2 * TC_LBO;
              const uint64_t bh = smem_desc_sbo(bs + ko, TC_SBO), bl = smem_desc_sbo(bs + Cfg::BMAT + ko, TC_SBO);
              const uint32_t acc0 = (c > 0 || kk > 0) ? 1u : 0u;
              mma_tf32(d1, arh, bh, Cfg::IDESC, acc0);
              mma_tf32(d1, arh, bl, Cfg::IDESC, 1u);
              mma_tf32(d1, arl, bh, Cfg::IDESC, 1u);
              mma_tf32(d2, aih, bh, Cfg::IDESC, acc0);
              mma_tf32(d2, aih, bl, Cfg::IDESC, 1u);
              mma_tf32(d2, ail, bh, Cfg::IDESC, 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             smem_u32(&bar.empty[slot]))
                         : "memory");
          }
          if (!ok) break;
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                           smem_u32(&bar.dfull[db]))
                       : "memory");
        }
      }
      // the last commits cover every MMA of this thread
      if (ok && TS > 0)
        t2_wait(&bar.dfull[(uint32_t)(TS - 1) % Cfg::DB], ((uint32_t)(TS - 1) / Cfg::DB) & 1, &bar, err);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    const int r = (warp & 3) * 32 + lane;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    int64_t ts = 0;
    bool ok = true;
    for (int64_t k = 0; k < K && ok; ++k) {
      const int64_t f = blockIdx.x + k * gridDim.x;
      for (int64_t t = 0; t < ntiles; ++t, ++ts) {
        const uint32_t tsu = (uint32_t)ts;
        const int db = (int)(tsu % Cfg::DB);
        ok = t2_wait(&bar.dfull[db], (tsu / Cfg::DB) & 1, &bar, err);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t d1 = tm + lane_base + (uint32_t)db * Cfg::DBUF, d2 = d1 + 64 * NCH;
        const int64_t t0 = tiles[t].t0, nt = tiles[t].nt;
        const bool any = tiles[t].ns > 0;
        const int64_t ro = r < nt ? (f * B + tgt[t0 + r]) * TC_C : -1;
#pragma unroll
        for (int h = 0; h < TC_C * NCH; h += 16) {
          // channels h .. h + 15 of the pass: chunk h / 32, its channels h % 32 + n
          float re[16], im[16], p[16];
          tmem_ld16(d1 + h, re);                 // K_r Q_r
          tmem_ld16(d2 + 32 * NCH + h, p);       // K_i Q_i
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
          for (int n = 0; n < 16; ++n) re[n] -= p[n];
          tmem_ld16(d1 + 32 * NCH + h, im);      // K_r Q_i
          tmem_ld16(d2 + h, p);                  // K_i Q_r
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
          for (int n = 0; n < 16; ++n) im[n] += p[n];
          if (h + 16 == TC_C * NCH) {
            // the accumulators of this buffer are read: the MMA warp may reuse it
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            mbar_arrive(&bar.dempty[db]);
          }
          if (ro >= 0) {
            float2* out = (h < TC_C ? Rh0 : Rh1) + ro + (h % TC_C);
#pragma unroll
            for (int n = 0; n < 16; n += 2)
              *reinterpret_cast<float4*>(out + n) =
                  any ? make_float4(re[n], im[n], re[n + 1], im[n + 1]) : make_float4(0.f, 0.f, 0.f, 0.f);
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tm), "r"(T2_COLS));
}

// ---------------------------------------------------------------------------
// Same pipeline, fed by a loader warp.  The producers of k_mac_top_tc2 wait on
// their own global loads (index rows and source spectra, one chunk ahead);
// here a loader warp copies, for every chunk, the tile's index block (16
// sources x tpad targets, contiguous in the tile's index table) and the
// chunk's source spectrum rows (256 bytes per source and 8-RHS chunk) into a
// ring of shared-memory stages, LSTG chunks ahead, in 16-byte asynchronous
// copies spread over its lanes, and the kernel spectrum rows (one buffer, or
// two where they fit) by TMA bulk copies.  The
// producers read everything from shared memory.  Roles: producers (warps
// 0-7), MMA lane (warp 8), loader lane (warp 9), epilogue (warps 10-13).
namespace {
constexpr int T3_PROD = 256;
constexpr int T3_MMA_WARP = 8;
constexpr int T3_LOAD_WARP = 9;
constexpr int T3_THREADS = 448;
constexpr int T3_LSTG = 8;                 // most loader stages (barrier arrays)
constexpr int T3_IBYTES = TC_KC * 128 * 4;   // index block of a chunk, at most 128 targets
constexpr int T3_QBYTES = TC_KC * TC_C * 8;  // source spectra of a chunk, one 8-RHS chunk
template <int NCH>
struct T3Cfg {
  static constexpr int LSTAGE = T3_IBYTES + NCH * T3_QBYTES;
};
struct T3Bar {
  uint64_t full[T2_STAGES], empty[T2_STAGES], dfull[2], dempty[2], rfull[2], rempty[2], lfull[T3_LSTG],
      lempty[T3_LSTG];
  uint32_t tmem_base;
  int abort;
  int nq;
};
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void arrive_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
}  // namespace

// dynamic shared memory: [nrow kernel rows of kbytes][STG B stages][LSTG
// loader stages][tile table][chunk table]
template <int NCH>
__global__ void __maxnreg__(128)
    k_mac_top_tc3(const float2* __restrict__ Qh0, const float2* __restrict__ Qh1, float2* __restrict__ Rh0,
                  float2* __restrict__ Rh1, const float2* __restrict__ Kh, int64_t B, int64_t O, int64_t nf,
                  int64_t ntiles, const int64_t* __restrict__ tgt_ptr, const int32_t* __restrict__ tgt,
                  const int64_t* __restrict__ src_ptr, const int32_t* __restrict__ src,
                  const int64_t* __restrict__ kidx_off, const int32_t* __restrict__ kidx, int kbytes, int nrow,
                  int lstg, int nq_cap, int* err) {
  extern __shared__ __align__(1024) unsigned char t3_smem[];
  __shared__ T3Bar bar;
  using Cfg = T2Cfg<NCH>;
  unsigned char* rows = t3_smem;
  unsigned char* Bs = t3_smem + nrow * kbytes;
  unsigned char* Ls = Bs + Cfg::STG * Cfg::BSTAGE;
  T2Tile* tiles = reinterpret_cast<T2Tile*>(Ls + lstg * T3Cfg<NCH>::LSTAGE);
  uint32_t* ctab = reinterpret_cast<uint32_t*>(tiles + ntiles);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t K = nf > blockIdx.x ? (nf - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  if (tid == 0) {
    for (int i = 0; i < Cfg::STG; ++i) {
      mbar_init(&bar.full[i], 128);
      mbar_init(&bar.empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bar.dfull[i], 1);
      mbar_init(&bar.dempty[i], 128);
      mbar_init(&bar.rfull[i], 1);
      mbar_init(&bar.rempty[i], T3_PROD);
    }
    for (int i = 0; i < lstg; ++i) {
      mbar_init(&bar.lfull[i], 32);
      mbar_init(&bar.lempty[i], 128);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    bar.abort = 0;
    int q = 0;
    for (int64_t t = 0; t < ntiles; ++t) {
      const int64_t ns = src_ptr[t + 1] - src_ptr[t], nt = tgt_ptr[t + 1] - tgt_ptr[t];
      tiles[t].koff = kidx_off[t];
      tiles[t].s0 = src_ptr[t];
      tiles[t].t0 = (int32_t)tgt_ptr[t];
      tiles[t].nt = (int32_t)nt;
      tiles[t].tpad = (int32_t)(((nt + 7) / 8) * 8);
      tiles[t].ns = (int32_t)ns;
      for (int64_t j0 = 0; j0 < ns && q < nq_cap; j0 += TC_KC) ctab[q++] = (uint32_t)((t << 16) | j0);
    }
    bar.nq = q;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&bar.tmem_base)),
                 "r"(T2_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tm = bar.tmem_base;
  const int64_t nq = bar.nq;
  const int64_t TS = K * ntiles;
  int* abar = &bar.abort;

  if (tid < T3_PROD) {
    // ------------------------------------------------------------ producers
    const int wg = tid >> 7, r = tid & 127;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    const int jB = (warp & 3) * 4 + (lane >> 3), chB = lane & 7;
    const int boff = (jB >> 2) * TC_LBO + (jB & 3) * 4 + chB * 16;
    int64_t g = wg;
    bool ok = true;
    for (int64_t k = 0; k < K && ok; ++k) {
      const int rb = nrow == 2 ? (int)(k & 1) : 0;
      const uint32_t rpar = (uint32_t)((nrow == 2 ? (k >> 1) : k) & 1);
      ok = t2_wait(&bar.rfull[rb], rpar, abar, err);
      if (!ok) break;
      const float2* Ks = reinterpret_cast<const float2*>(rows + rb * kbytes);
      for (; g < (k + 1) * nq; g += 2) {
        const uint32_t gu = (uint32_t)g;
        const int ls = (int)(gu % (uint32_t)lstg);
        ok = t2_wait(&bar.lfull[ls], (gu / (uint32_t)lstg) & 1, abar, err);
        if (!ok) break;
        const uint32_t e = ctab[g - k * nq];
        const T2Tile& T = tiles[e >> 16];
        const int j0 = (int)(e & 0xFFFFu);
        const unsigned char* st = Ls + ls * T3Cfg<NCH>::LSTAGE;
        const int32_t* Is = reinterpret_cast<const int32_t*>(st);
        const float2* Qs = reinterpret_cast<const float2*>(st + T3_IBYTES);
        int32_t idc[TC_KC];
        float2 qc[4 * NCH];
#pragma unroll
        for (int j = 0; j < TC_KC; ++j) idc[j] = (r < T.tpad && j0 + j < T.ns) ? Is[j * T.tpad + r] : -1;
        const bool qv = j0 + jB < T.ns;
#pragma unroll
        for (int u = 0; u < 4; ++u) qc[u] = qv ? Qs[jB * TC_C + chB + 8 * u] : make_float2(0.f, 0.f);
        if (NCH == 2) {
#pragma unroll
          for (int u = 0; u < 4; ++u)
            qc[4 + u] = qv ? Qs[TC_KC * TC_C + jB * TC_C + chB + 8 * u] : make_float2(0.f, 0.f);
        }
        mbar_arrive(&bar.lempty[ls]);   // the stage is read
        const int slot = (int)(gu % Cfg::STG);
        if (gu >= (uint32_t)Cfg::STG) {
          ok = t2_wait(&bar.empty[slot], ((gu / Cfg::STG) - 1) & 1, abar, err);
          if (!ok) break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        {
          const uint32_t ta = tm + lane_base + T2_A0 + (uint32_t)slot * 4 * TC_KC;
#pragma unroll
          for (int hh = 0; hh < TC_KC; hh += 8) {
            float arh[8], arl[8], aih[8], ail[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const float2 kv = idc[hh + j] >= 0 ? Ks[idc[hh + j]] : make_float2(0.f, 0.f);
              arh[j] = tf32_hi(kv.x);
              arl[j] = kv.x - arh[j];
              aih[j] = tf32_hi(kv.y);
              ail[j] = kv.y - aih[j];
            }
            tmem_st8(ta + 0 * TC_KC + hh, arh);
            tmem_st8(ta + 1 * TC_KC + hh, arl);
            tmem_st8(ta + 2 * TC_KC + hh, aih);
            tmem_st8(ta + 3 * TC_KC + hh, ail);
          }
        }
        {
          float* bb = reinterpret_cast<float*>(Bs + slot * Cfg::BSTAGE + boff);
#pragma unroll
          for (int u = 0; u < 4 * NCH; ++u) {
            const float rh = tf32_hi(qc[u].x), ih = tf32_hi(qc[u].y);
            bb[(u * TC_SBO) / 4] = rh;
            bb[((4 * NCH + u) * TC_SBO) / 4] = ih;
            bb[(Cfg::BMAT + u * TC_SBO) / 4] = qc[u].x - rh;
            bb[(Cfg::BMAT + (4 * NCH + u) * TC_SBO) / 4] = qc[u].y - ih;
          }
        }
        asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        mbar_arrive(&bar.full[slot]);
      }
      if (!ok) break;
      mbar_arrive(&bar.rempty[rb]);   // this thread is done with the row buffer
    }
  } else if (warp == T3_MMA_WARP) {
    // ------------------------------------------------------------ MMA warp
    if (lane == 0) {
      bool ok = true;
      int64_t g = 0, ts = 0;
      for (int64_t k = 0; k < K && ok; ++k) {
        for (int64_t t = 0; t < ntiles && ok; ++t, ++ts) {
          const uint32_t tsu = (uint32_t)ts;
          const int db = (int)(tsu % Cfg::DB);
          if (tsu >= (uint32_t)Cfg::DB) {
            ok = t2_wait(&bar.dempty[db], ((tsu / Cfg::DB) - 1) & 1, abar, err);
            if (!ok) break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
          const int64_t nch = (tiles[t].ns + TC_KC - 1) / TC_KC;
          const uint32_t d1 = tm + (uint32_t)db * Cfg::DBUF, d2 = d1 + 64 * NCH;
          for (int64_t c = 0; c < nch; ++c, ++g) {
            const uint32_t gu = (uint32_t)g;
            const int slot = (int)(gu % Cfg::STG);
            ok = t2_wait(&bar.full[slot], (gu / Cfg::STG) & 1, abar, err);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t a0 = tm + T2_A0 + (uint32_t)slot * 4 * TC_KC;
            const uint32_t bs = smem_u32(Bs + slot * Cfg::BSTAGE);
#pragma unroll
            for (int kk = 0; kk < TC_KC / 8; ++kk) {
              const uint32_t arh = a0 + 0 * TC_KC + kk * 8, arl = a0 + 1 * TC_KC + kk * 8;
              const uint32_t aih = a0 + 2 * TC_KC + kk * 8, ail = a0 + 3 * TC_KC + kk * 8;
              const uint32_t ko = (uint32_t)kk * 2 * TC_LBO;
              const uint64_t bh = smem_desc_sbo(bs + ko, TC_SBO), bl = smem_desc_sbo(bs + Cfg::BMAT + ko, TC_SBO);
              const uint32_t acc0 = (c > 0 || kk > 0) ? 1u : 0u;
              mma_tf32(d1, arh, bh, Cfg::IDESC, acc0);
              mma_tf32(d1, arh, bl, Cfg::IDESC, 1u);
              mma_tf32(d1, arl, bh, Cfg::IDESC, 1u);
              mma_tf32(d2, aih, bh, Cfg::IDESC, acc0);
              mma_tf32(d2, aih, bl, Cfg::IDESC, 1u);
              mma_tf32(d2, ail, bh, Cfg::IDESC, 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             smem_u32(&bar.empty[slot]))
                         : "memory");
          }
          if (!ok) break;
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                           smem_u32(&bar.dfull[db]))
                       : "memory");
        }
      }
      if (ok && TS > 0)
        t2_wait(&bar.dfull[(uint32_t)(TS - 1) % Cfg::DB], ((uint32_t)(TS - 1) / Cfg::DB) & 1, abar, err);
    }
    __syncwarp();
  } else if (warp == T3_LOAD_WARP) {
    // ------------------------------------------------------------ loader
    // lane 0 waits on the ring and copies the kernel rows (TMA bulk copies);
    // the 32 lanes copy each chunk's index block and source spectra in
    // 16-byte asynchronous copies and each signals lfull when its own
    // copies have landed (lfull counts 32 arrivals)
    bool ok = true;
    int64_t g = 0;
    const uint32_t rbytes = (uint32_t)(O * 8);
    for (int64_t k = 0; k < K && ok; ++k) {
      const int64_t f = blockIdx.x + k * gridDim.x;
      const int rb = nrow == 2 ? (int)(k & 1) : 0;
      if (k >= nrow) {
        const uint32_t use = (uint32_t)(nrow == 2 ? (k >> 1) : k);   // earlier uses of this buffer
        int w = 1;
        if (lane == 0) w = t2_wait(&bar.rempty[rb], (use - 1) & 1, abar, err) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, w, 0) != 0;
        if (!ok) break;
      }
      if (lane == 0) {
        const unsigned char* srow = reinterpret_cast<const unsigned char*>(Kh + f * O);
        const uint32_t dst = smem_u32(rows + rb * kbytes);
        arrive_tx(&bar.rfull[rb], rbytes);
        for (uint32_t off = 0; off < rbytes; off += T2_PIECE) {
          const uint32_t n = rbytes - off < (uint32_t)T2_PIECE ? rbytes - off : (uint32_t)T2_PIECE;
          bulk_g2s(dst + off, srow + off, n, &bar.rfull[rb]);
        }
      }
      for (int64_t q = 0; q < nq; ++q, ++g) {
        const uint32_t gu = (uint32_t)g;
        const int ls = (int)(gu % (uint32_t)lstg);
        if (gu >= (uint32_t)lstg) {
          int w = 1;
          if (lane == 0) w = t2_wait(&bar.lempty[ls], ((gu / (uint32_t)lstg) - 1) & 1, abar, err) ? 1 : 0;
          ok = __shfl_sync(0xffffffffu, w, 0) != 0;
          if (!ok) break;
        }
        const uint32_t e = ctab[q];
        const T2Tile& T = tiles[e >> 16];
        const int j0 = (int)(e & 0xFFFFu);
        const int nsrc = T.ns - j0 < TC_KC ? T.ns - j0 : TC_KC;
        const int iseg = nsrc * T.tpad / 4;   // 16-byte pieces of the index block
        const uint32_t st = smem_u32(Ls + ls * T3Cfg<NCH>::LSTAGE);
        const int32_t yl = lane < nsrc ? __ldg(src + T.s0 + j0 + lane) : 0;
        const unsigned char* ksrc = reinterpret_cast<const unsigned char*>(kidx + T.koff + (int64_t)j0 * T.tpad);
        for (int sg = lane; sg < iseg; sg += 32) cp_async16(st + sg * 16, ksrc + sg * 16);
        const int qseg = nsrc * 16;           // 16-byte pieces of the source rows of one 8-RHS chunk
        for (int it = 0; it < 8; ++it) {
          const int sg = it * 32 + lane, j = sg >> 4, part = sg & 15;
          const int64_t yj = __shfl_sync(0xffffffffu, yl, j & 31);
          if (sg < qseg) {
            const int64_t o = (f * B + yj) * TC_C + part * 2;
            cp_async16(st + T3_IBYTES + sg * 16, Qh0 + o);
            if (NCH == 2) cp_async16(st + T3_IBYTES + T3_QBYTES + sg * 16, Qh1 + o);
          }
        }
        asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(smem_u32(&bar.lfull[ls]))
                     : "memory");
      }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    const int r = (warp & 3) * 32 + lane;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    int64_t ts = 0;
    bool ok = true;
    for (int64_t k = 0; k < K && ok; ++k) {
      const int64_t f = blockIdx.x + k * gridDim.x;
      for (int64_t t = 0; t < ntiles; ++t, ++ts) {
        const uint32_t tsu = (uint32_t)ts;
        const int db = (int)(tsu % Cfg::DB);
        ok = t2_wait(&bar.dfull[db], (tsu / Cfg::DB) & 1, abar, err);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t d1 = tm + lane_base + (uint32_t)db * Cfg::DBUF, d2 = d1 + 64 * NCH;
        const int64_t t0 = tiles[t].t0, nt = tiles[t].nt;
        const bool any = tiles[t].ns > 0;
        const int64_t ro = r < nt ? (f * B + tgt[t0 + r]) * TC_C : -1;
#pragma unroll
        for (int h = 0; h < TC_C * NCH; h += 16) {
          float re[16], im[16], p[16];
          tmem_ld16(d1 + h, re);
          tmem_ld16(d2 + 32 * NCH + h, p);
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
          for (int n = 0; n < 16; ++n) re[n] -= p[n];
          tmem_ld16(d1 + 32 * NCH + h, im);
          tmem_ld16(d2 + h, p);
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
          for (int n = 0; n < 16; ++n) im[n] += p[n];
          if (h + 16 == TC_C * NCH) {
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            mbar_arrive(&bar.dempty[db]);
          }
          if (ro >= 0) {
            float2* out = (h < TC_C ? Rh0 : Rh1) + ro + (h % TC_C);
#pragma unroll
            for (int n = 0; n < 16; n += 2)
              *reinterpret_cast<float4*>(out + n) =
                  any ? make_float4(re[n], im[n], re[n + 1], im[n + 1]) : make_float4(0.f, 0.f, 0.f, 0.f);
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tm), "r"(T2_COLS));
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
  static SmemAttr attr;
  smem_attr_once(k_mac_top_tc, (int)smem, attr.v);
  for (int64_t fs = 0; fs < nf; fs += 65535) {
    const int64_t nfc = nf - fs < 65535 ? nf - fs : 65535;
    dim3 grid((unsigned)ntiles, (unsigned)nfc);
    k_mac_top_tc<<<grid, 128, (size_t)smem, s>>>(Qh, Rh, Kh, B, O, nf, tgt_ptr, tgt, src_ptr, src, kidx_off, kidx,
                                                 fs, (int)kbytes, err);
  }
  return true;
}

// The persistent kernel takes tiles of at most 128 targets with any source
// lists, 32 channels per chunk, an even number of offsets (kernel rows are
// copied by TMA in 16-byte units) below 32,768 (offset ids are read as int16
// from the chunk-major index blocks [chunk][tpad][16] of make_index16), and
// shared memory for two kernel rows, the
// B stages and the tile and chunk tables (nq = sum over tiles of
// ceil(sources / 16); at most 65,536 sources per tile, as a chunk-table entry
// holds tile and first source in 16 bits each).  Returns false when it does
// not apply.
static int64_t tc2_smem_bytes(int64_t O, int nch, int64_t ntiles, int64_t nq) {
  const int64_t kbytes = ((O * 8 + 1023) / 1024) * 1024;
  // at least 120 KB: one CTA (one 512-column TMEM allocation) per SM
  return std::max<int64_t>(2 * kbytes + (nch == 1 ? 4 * T2Cfg<1>::BSTAGE : 3 * T2Cfg<2>::BSTAGE) +
                               ntiles * (int64_t)sizeof(T2Tile) + nq * 4,
                           120 * 1024);
}

bool mac_top_tc2_fits(int C, int max_tile_targets, int64_t O, int64_t nq, int64_t ntiles, int nch) {
  return C == TC_C && (nch == 1 || nch == 2) && max_tile_targets > 8 && max_tile_targets <= 128 && O > 0 &&
         O <= 32767 &&
         (O % 2) == 0 && ntiles > 0 && ntiles < 65536 && nq > 0 && tc2_smem_bytes(O, nch, ntiles, nq) <= 220 * 1024;
}

// nch = 2: two 8-right-hand-side chunks in one pass (Qh[1], Rh[1] used),
// B operands of 128 rows and N = 128 MMAs.
bool launch_mac_top_tc2(const float2* const* Qh, float2* const* Rh, int nch, const float2* Kh, int64_t B, int C,
                        int64_t O, int64_t nf, int64_t ntiles, int max_tile_targets, const int64_t* tgt_ptr,
                        const int32_t* tgt, const int64_t* src_ptr, const int32_t* src, const int64_t* kidx_off,
                        const int16_t* kidx, int64_t nq, int* err, cudaStream_t s) {
  if (!mac_top_tc2_fits(C, max_tile_targets, O, nq, ntiles, nch) || nf <= 0) return false;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return false;
  const int64_t kbytes = ((O * 8 + 1023) / 1024) * 1024;
  const int64_t smem = tc2_smem_bytes(O, nch, ntiles, nq);
  const unsigned grid = (unsigned)std::min<int64_t>(nf, nsm);
  if (nch == 1) {
    static SmemAttr attr;
    smem_attr_once(k_mac_top_tc2<1>, (int)smem, attr.v);
    k_mac_top_tc2<1><<<grid, T2_THREADS, (size_t)smem, s>>>(Qh[0], nullptr, Rh[0], nullptr, Kh, B, O, nf, ntiles,
                                                            tgt_ptr, tgt, src_ptr, src, kidx_off, kidx, (int)kbytes,
                                                            (int)nq, err);
  } else {
    static SmemAttr attr;
    smem_attr_once(k_mac_top_tc2<2>, (int)smem, attr.v);
    k_mac_top_tc2<2><<<grid, T2_THREADS, (size_t)smem, s>>>(Qh[0], Qh[1], Rh[0], Rh[1], Kh, B, O, nf, ntiles,
                                                            tgt_ptr, tgt, src_ptr, src, kidx_off, kidx, (int)kbytes,
                                                            (int)nq, err);
  }
  return true;
}


// The loader-fed kernel: one or two kernel-row buffers (two where they fit
// in 220 KB with the B stages, loader stages and tables), the same tile
// limits as k_mac_top_tc2.
static int64_t tc3_smem_bytes(int64_t O, int nch, int64_t ntiles, int64_t nq, int nrow, int lstg) {
  const int64_t kbytes = ((O * 8 + 1023) / 1024) * 1024;
  const int64_t b = nch == 1 ? T2Cfg<1>::STG * T2Cfg<1>::BSTAGE : T2Cfg<2>::STG * T2Cfg<2>::BSTAGE;
  const int64_t l = lstg * (nch == 1 ? T3Cfg<1>::LSTAGE : T3Cfg<2>::LSTAGE);
  // at least 120 KB, so that a second CTA (and a second 512-column TMEM
  // allocation) never fits on an SM
  return std::max<int64_t>(nrow * kbytes + b + l + ntiles * (int64_t)sizeof(T2Tile) + nq * 4, 120 * 1024);
}

// kernel-row buffers and loader stages: as many as fit in 220 KB, preferring
// two row buffers, then up to 8 loader stages (at least 4)
static void tc3_shape(int64_t O, int nch, int64_t ntiles, int64_t nq, int* nrow, int* lstg) {
  *nrow = 0;
  *lstg = 0;
  for (int r = 2; r >= 1 && *nrow == 0; --r)
    for (int l = T3_LSTG; l >= 4; --l)
      if (tc3_smem_bytes(O, nch, ntiles, nq, r, l) <= 220 * 1024) {
        *nrow = r;
        *lstg = l;
        break;
      }
}

bool mac_top_tc3_fits(int C, int max_tile_targets, int64_t O, int64_t nq, int64_t ntiles, int nch) {
  return C == TC_C && (nch == 1 || nch == 2) && max_tile_targets > 8 && max_tile_targets <= 128 && O > 0 &&
         (O % 2) == 0 && O * 8 < (1 << 20) && ntiles > 0 && ntiles < 65536 && nq > 0 &&
         [&] {
           int r, l;
           tc3_shape(O, nch, ntiles, nq, &r, &l);
           return r > 0;
         }();
}

bool launch_mac_top_tc3(const float2* const* Qh, float2* const* Rh, int nch, const float2* Kh, int64_t B, int C,
                        int64_t O, int64_t nf, int64_t ntiles, int max_tile_targets, const int64_t* tgt_ptr,
                        const int32_t* tgt, const int64_t* src_ptr, const int32_t* src, const int64_t* kidx_off,
                        const int32_t* kidx, int64_t nq, int* err, cudaStream_t s) {
  if (!mac_top_tc3_fits(C, max_tile_targets, O, nq, ntiles, nch) || nf <= 0) return false;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return false;
  int nrow = 0, lstg = 0;
  tc3_shape(O, nch, ntiles, nq, &nrow, &lstg);
  const int64_t kbytes = ((O * 8 + 1023) / 1024) * 1024;
  const int64_t smem = tc3_smem_bytes(O, nch, ntiles, nq, nrow, lstg);
  const unsigned grid = (unsigned)std::min<int64_t>(nf, nsm);
  if (nch == 1) {
    static SmemAttr attr;
    smem_attr_once(k_mac_top_tc3<1>, (int)smem, attr.v);
    k_mac_top_tc3<1><<<grid, T3_THREADS, (size_t)smem, s>>>(Qh[0], nullptr, Rh[0], nullptr, Kh, B, O, nf, ntiles,
                                                            tgt_ptr, tgt, src_ptr, src, kidx_off, kidx, (int)kbytes,
                                                            nrow, lstg, (int)nq, err);
  } else {
    static SmemAttr attr;
    smem_attr_once(k_mac_top_tc3<2>, (int)smem, attr.v);
    k_mac_top_tc3<2><<<grid, T3_THREADS, (size_t)smem, s>>>(Qh[0], Qh[1], Rh[0], Rh[1], Kh, B, O, nf, ntiles,
                                                            tgt_ptr, tgt, src_ptr, src, kidx_off, kidx, (int)kbytes,
                                                            nrow, lstg, (int)nq, err);
  }
  return true;
}
}  // namespace efie
