// C ABI of the GB300 fast EFIE library: setup orchestration, the matvec
// pipeline (charges, anterpolation, transfers, translations, interpolation, near field) and the batched GMRES / FGMRES driver.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <functional>
#include <cmath>
#include <complex>
#include <cstring>
#include <memory>
#include <random>
#include <string>
#include <vector>

#include "../../include/efie.h"
#include "common.cuh"
#include "device_api.cuh"
#include "plan.hpp"

namespace efie {
int upload_rhs_rule(const double* q6);
struct Net;
int nn_param_count();
void nn_init_params(std::vector<float>& p, uint64_t seed);
void nn_setup(Net& net, int64_t N, const std::vector<int32_t>& nbr, const std::vector<float>& sgn,
              const std::vector<float>& lnorm, const std::vector<float>& params, bool training);
void nn_free(Net& net);
void nn_forward(Net& net, const double2* r, double2* z, bool training, cudaStream_t s);
void nn_backward(Net& net, const double2* z, const double2* e, double2* gbuf, cudaStream_t s);
void nn_backward_g(Net& net, const double2* gz, cudaStream_t s);
void nn_zero_grad(Net& net, cudaStream_t s);
void nn_adam(Net& net, float lr, float gscale, cudaStream_t s);
void nn_read_params(Net& net, std::vector<float>& out);
void nn_read_grads(Net& net, std::vector<float>& out);
void nn_loss_terms(Net& net, double* num, double* den);
Net* nn_new();
void nn_delete(Net* n);
}

using namespace efie;

namespace {

thread_local std::string g_last_error = "";

void cuda_check(cudaError_t e, const char* what) {
  if (e != cudaSuccess)
    throw EfieError{e == cudaErrorMemoryAllocation ? EFIE_ENOMEM : EFIE_ECUDA,
                    std::string(what) + ": " + cudaGetErrorString(e)};
}

// device allocation tracker: every allocation of a handle, with its size, so
// that released buffers leave the device_mem_limit budget
struct DevMem {
  std::vector<std::pair<void*, int64_t>> ptrs;
  int64_t bytes = 0, limit = 0;
  template <typename T>
  T* alloc(int64_t n) {
    if (n <= 0) n = 1;
    int64_t b = n * (int64_t)sizeof(T);
    if (limit > 0 && bytes + b > limit)
      throw EfieError{EFIE_ENOMEM, "device_mem_limit exceeded (" + std::to_string(bytes + b) + " bytes)"};
    void* p = nullptr;
    cuda_check(cudaMalloc(&p, (size_t)b), "cudaMalloc");
    ptrs.push_back({p, b});
    bytes += b;
    return (T*)p;
  }
  template <typename T>
  T* upload(const std::vector<T>& v) {
    T* p = alloc<T>((int64_t)v.size());
    if (!v.empty()) cuda_check(cudaMemcpy(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice), "upload");
    return p;
  }
  void release(void* p) {
    if (!p) return;
    for (size_t i = 0; i < ptrs.size(); ++i)
      if (ptrs[i].first == p) {
        cudaFree(p);
        bytes -= ptrs[i].second;
        ptrs.erase(ptrs.begin() + (int64_t)i);
        return;
      }
  }
  ~DevMem() {
    for (auto& q : ptrs) cudaFree(q.first);
  }
};

template <typename R>
struct FarSet {
  bool built = false;
  R *mr = nullptr, *mt = nullptr;  // moments by basis function (interpolation)
  R *gr = nullptr, *gt = nullptr;  // the same moments by grid point (anterpolation)
  struct Lev {
    cpx_t<R>* Mf = nullptr;
    cpx_t<R>* Mb = nullptr;
    R *CL = nullptr, *CR = nullptr, *CLt = nullptr, *CRt = nullptr;
    cpx_t<R>* Kh = nullptr;
    cpx_t<R>* KH[6] = {};  // dyadic factorization: Hessian spectra, ab = 00, 01, 02, 11, 12, 22
  };
  std::vector<Lev> lv;
  int Rc = 0;
  std::vector<cpx_t<R>*> q, r;
  cpx_t<R>*tmp1 = nullptr, *tmp2 = nullptr, *Qh = nullptr, *Rh = nullptr;
  // second chunk of a chunk pair (one translation pass per level over 16
  // right-hand sides): its level grids q2[], r2[], and spectra buffers for its
  // sources (Qt2) and results (Rt2)
  std::vector<cpx_t<R>*> q2, r2;
  cpx_t<R>*Qt2 = nullptr, *Rt2 = nullptr;
  // dyadic factorization: level grids and a spectrum buffer of the Hessian
  // translation, for chunks of up to Rd right-hand sides
  int Rd = 0;
  std::vector<cpx_t<R>*> rd;
  cpx_t<R>* Rdh = nullptr;
};

struct LevDev {
  int64_t B = 0;
  int64_t* il_ptr = nullptr;
  int32_t* il_src = nullptr;
  int32_t* il_off = nullptr;
  int32_t* offsets = nullptr;
  int64_t* parent = nullptr;
  int8_t* bits = nullptr;
  int64_t* child_ptr = nullptr;
  int64_t nfar = 0, O = 0;
  // translation tiles
  int64_t ntiles = 0;
  int max_tile = 0;
  int64_t nq = 0;        // chunks of 16 sources summed over the tiles
  // tensor-core tiles of an interaction-list level (128 targets, union sources)
  int64_t tct_ntiles = 0, tct_nq = 0;
  int tct_max = 0;
  int64_t *tct_tgt_ptr = nullptr, *tct_src_ptr = nullptr, *tct_kidx_off = nullptr;
  int32_t *tct_tgt = nullptr, *tct_src = nullptr, *tct_kidx = nullptr;
  int64_t *tile_tgt_ptr = nullptr, *tile_src_ptr = nullptr, *tile_kidx_off = nullptr;
  int32_t *tile_tgt = nullptr, *tile_src = nullptr, *tile_kidx = nullptr;
  // the same index tiles for the persistent tensor-core kernel: int16 ids in
  // chunk-major blocks [chunk of 16 sources][tpad targets][16] per tile (null
  // where an id does not fit in int16)
  int64_t *tile_k16_off = nullptr, *tct_k16_off = nullptr;
  int16_t *tile_k16 = nullptr, *tct_k16 = nullptr;
  // sibling-shared transfers between this (child) level and its parents:
  // g1 = (parent, b_x, b_y) groups of children, g2 = (parent, b_x) groups
  int64_t ng1 = 0, ng2 = 0;
  int64_t *uz_s0 = nullptr, *uz_s1 = nullptr, *uy_s0 = nullptr, *uy_s1 = nullptr, *ux_s0 = nullptr,
          *ux_s1 = nullptr;
  int8_t *uz_b0 = nullptr, *uz_b1 = nullptr, *uy_b0 = nullptr, *uy_b1 = nullptr, *ux_b0 = nullptr,
         *ux_b1 = nullptr;
  int64_t *dx_src = nullptr, *dy_src = nullptr, *dz_src = nullptr;  // downward: g2 -> parent, g1 -> g2, child -> g1
  int8_t *dx_sel = nullptr, *dy_sel = nullptr;                      // [G][3]
  // leaves of the tree on this level (all boxes of level D in a uniform tree;
  // several levels in a nonuniform one): global leaf ids [leaf0, leaf0 + nleaf),
  // their box indices (null when they are the level's boxes in order), and the
  // gather-list offsets of their grid points
  int64_t leaf0 = 0, nleaf = 0;
  int32_t* leaf_box = nullptr;
  int32_t *gptr_r = nullptr, *gptr_t = nullptr;
};

std::complex<double> jk_of(double k) { return std::complex<double>(0.0, k); }

}  // namespace

namespace {
// kernel classes for the profiling facility
enum KClass {
  K_VEC = 0, K_ANTERP, K_UP, K_FWD, K_MAC, K_INV, K_DOWN, K_INTERP, K_NEAR_A, K_NEAR_V, K_KRYLOV, K_MAC_TOP,
  K_PRECOND, K_MAC_TOP_TC, K_MAC_TC, K_NCLASS
};
const char* kclass_name[K_NCLASS] = {"vector",   "anterpolation", "upward",  "forward_fft", "translation_mac",
                                     "inverse_fft", "downward",   "interpolation", "near_A", "near_V", "krylov",
                                     "translation_mac_top", "precond", "translation_mac_top_tc",
                                     "translation_mac_tc"};
struct Prof {
  bool on = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev;
  int64_t launches[K_NCLASS] = {0};
  void clear() {
    for (auto& e : ev) {
      cudaEventDestroy(e.second.first);
      cudaEventDestroy(e.second.second);
    }
    ev.clear();
    for (auto& l : launches) l = 0;
  }
  ~Prof() { clear(); }
};
}  // namespace

// Copy streams, events and double-buffered device staging for
// efie_matvec_host (created on first use).
struct HostPipe {
  bool ready = false;
  int rc = 0;                        // right-hand sides per staging slot
  cudaStream_t s_in = nullptr, s_out = nullptr;
  cudaEvent_t ev_start = nullptr, ev_end = nullptr;
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_comp[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
  double2 *xs[2] = {nullptr, nullptr}, *ys[2] = {nullptr, nullptr};
  ~HostPipe() {
    for (int b = 0; b < 2; ++b) {
      if (ev_in[b]) cudaEventDestroy(ev_in[b]);
      if (ev_comp[b]) cudaEventDestroy(ev_comp[b]);
      if (ev_out[b]) cudaEventDestroy(ev_out[b]);
    }
    if (ev_start) cudaEventDestroy(ev_start);
    if (ev_end) cudaEventDestroy(ev_end);
    if (s_in) cudaStreamDestroy(s_in);
    if (s_out) cudaStreamDestroy(s_out);
  }
};

struct efie_handle {
  Prof prof;
  HostPipe pipe;
  // learned preconditioner
  efie::Net* net = nullptr;
  bool net_training = false;
  std::vector<float> net_params;
  std::vector<int32_t> g_nbr;
  std::vector<float> g_sgn, g_len;
  ~efie_handle() {
    if (net) efie::nn_delete(net);
    if (err_host) cudaFreeHost(err_host);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (ev_far) cudaEventDestroy(ev_far);
    if (s_near) cudaStreamDestroy(s_near);
    if (s_far) cudaStreamDestroy(s_far);
  }
  int64_t n_launches = 0;
  double setup_s[4] = {0, 0, 0, 0};  // efie_setup phases (efie_setup_times)
  Plan plan;
  efie_options opt{};
  int precision = EFIE_FP64;
  std::string err;
  int device = 0;
  DevMem mem;
  // geometry
  double* dV = nullptr;
  int32_t* dT = nullptr;
  double* darea = nullptr;
  int32_t* dtri_pm = nullptr;
  int32_t* dfree_pm = nullptr;
  // orders
  int32_t *d_rwg_perm = nullptr, *d_rwg_box = nullptr, *d_tri_box = nullptr, *d_rwg_tri_sorted = nullptr;
  int64_t *d_box_rwg_ptr = nullptr, *d_box_tri_ptr = nullptr;
  int32_t* d_tri_rwg = nullptr;
  // scalar (charge) part of the factorization: star (Sec. VI-A) pulses on the
  // triangles, or direct (Sec. VI-B) divergence moments of the RWGs
  bool direct = false;
  bool dyadic = false;   // dyadic factorization (Sec. VI-C): direct-form near field and moments, plus the
                         // Hessian translation of the three vector components
  double2* wd = nullptr; // dyadic: scratch for the scalar output of the Hessian grids' interpolation
  int64_t n_sc = 0;                  // scalar items: triangles (star) or RWGs (direct)
  const int64_t* d_sc_box_ptr = nullptr;  // items of each leaf
  const int32_t* d_sc_box = nullptr;      // leaf of each item
  // box of each sorted function on its leaf's level (RWG, triangle, scalar item)
  int32_t *d_rwg_lbox = nullptr, *d_tri_lbox = nullptr;
  const int32_t* d_sc_lbox = nullptr;
  const int64_t* d_blkS_off = nullptr;    // near blocks of the scalar part (V, or Phi in A's layout)
  int8_t* d_tri_sgn = nullptr;
  // moments structure (shared by precisions)
  int32_t *mr_base = nullptr, *mr_ext = nullptr, *mt_base = nullptr, *mt_ext = nullptr;
  int64_t *mr_off = nullptr, *mt_off = nullptr;
  // near
  NearDev nd{};
  int64_t *d_near_ptr = nullptr, *d_blkA_off = nullptr, *d_blkV_off = nullptr;
  int32_t* d_near_src = nullptr;
  // far
  std::vector<LevDev> lev;
  FarSet<double> f64;
  FarSet<float> f32;
  int mac_variant = 0;   // translation (autotuner knob): 0 auto (tensor cores on the top level, persistent
                         // form, else 3, else 2; chunk pairs also take the interaction-list levels on
                         // tensor cores), 1 register tiles, 2 CUDA-core shared-memory staged, 3 tensor
                         // cores with one CTA per (tile, frequency), 4 as 0 but chunk pairs keep the
                         // interaction-list levels on CUDA cores, 5 as 0 with the loader-fed persistent form
  int* err_host = nullptr;  // host-mapped flag that device waits set when they run out
  int* err_dev = nullptr;
  int near_variant = 0;  // mixed near field (autotuner knob): 0 x staged in shared memory by
                         // double-buffered asynchronous copies, one thread per row and 8 RHS; 1 x
                         // through L1; 2 x staged by the block between barriers, 4 RHS per thread;
                         // 3 as 0 with an mbarrier ring filled by a copy warp
  int fft_variant = 3;   // transform schedule (autotuner knob): 0 line passes; 1 forward y and z passes
                         // fused per slab where they apply (FP32, 32 channels); 2 forward and inverse
                         // fused; 3 (default) both fused on levels of 9 splines per axis only
  // work vectors (FP64, sorted) and their double-float splits
  int Rw = 0;
  double2 *xs = nullptr, *rho = nullptr, *yA = nullptr, *w = nullptr;
  // near field on a second stream, overlapping the far field: its own outputs
  // (added in the final combination), fork / join events
  double2 *yAn = nullptr, *wn = nullptr;
  cudaStream_t s_near = nullptr;
  cudaStream_t s_far = nullptr;   // far field, highest priority, so its kernels go first
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_far = nullptr;
  float4 *xs4 = nullptr, *rho4 = nullptr;
  float2 *xsf = nullptr, *rhof = nullptr;   // FP32 copies for the far field
  bool near_df = false;   // near matrices stored as double-float pairs
};

namespace {
void net_activate(efie_handle* h, const std::vector<float>& params, bool training);
bool read_weights(const char* path, std::vector<float>& p);

// RAII scope around the launches of one kernel class: counts launches and,
// while profiling is on, records an event pair on the launching stream.
struct KScope {
  efie_handle* h;
  int cls;
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
  KScope(efie_handle* h_, int cls_, cudaStream_t s_, int nlaunch) : h(h_), cls(cls_), s(s_) {
    h->n_launches += nlaunch;
    if (h->prof.on) {
      h->prof.launches[cls] += nlaunch;
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      cudaEventRecord(a, s);
    }
  }
  ~KScope() {
    if (a) {
      cudaEventRecord(b, s);
      h->prof.ev.push_back({cls, {a, b}});
    }
  }
};

void set_err(efie_handle* h, const EfieError& e) {
  if (h) h->err = e.msg;
  g_last_error = e.msg;
}

efie_options defaults(const efie_options* o) {
  efie_options d{};
  if (o) d = *o;
  if (d.gmres_restart <= 0) d.gmres_restart = 100;
  if (d.max_iters <= 0) d.max_iters = 1000;
  if (d.precision != EFIE_MIXED) d.precision = EFIE_FP64;
  return d;
}

void check_mesh(const efie_mesh* mesh) {
  if (!mesh || !mesh->xyz || !mesh->tri || mesh->n_vertices < 4 || mesh->n_triangles < 4)
    throw EfieError{EFIE_EINVAL, "invalid mesh"};
}

void collapsed_rule(int n, std::vector<double>& out) {
  std::vector<double> x, w;
  gauss_legendre01(n, x, w);
  out.assign(3 * n * n, 0.0);
  int q = 0;
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b, ++q) {
      out[q] = x[a];
      out[n * n + q] = x[b] * (1.0 - x[a]);
      out[2 * n * n + q] = w[a] * w[b] * (1.0 - x[a]);
    }
}

// ------------------------------------------------------------- far setup
template <typename R>
void build_far(efie_handle* h, FarSet<R>& F, cudaStream_t s) {
  Plan& P = h->plan;
  DevMem& M = h->mem;
  // moments
  // RWG moments interleaved by entry on the device: [e][3] per basis function
  std::vector<R> mr(P.mom_rwg.data.size());
  {
    const MomentBlocks& MB = P.mom_rwg;
    const int64_t n = (int64_t)MB.off.size() - 1;
    for (int64_t i = 0; i < n; ++i) {
      const int64_t o = MB.off[i], ne = (MB.off[i + 1] - o) / 3;
      for (int64_t e = 0; e < ne; ++e)
        for (int d = 0; d < 3; ++d) mr[o + 3 * e + d] = (R)MB.data[o + d * ne + e];
    }
  }
  const MomentBlocks& MS = h->direct ? P.mom_div : P.mom_tri;   // scalar-part moments
  std::vector<R> mt(MS.data.begin(), MS.data.end());
  F.mr = M.upload(mr);
  F.mt = M.upload(mt);
  F.gr = M.alloc<R>((int64_t)mr.size() / 3 * 4);
  F.gt = M.alloc<R>((int64_t)mt.size() * 2);
  for (int ell = P.D; ell >= P.top; --ell) {
    // gather lists of the leaves of every level (the moment entries are the
    // same in both precisions, so the offsets are built once)
    LevDev& LD = h->lev[ell - P.top];
    if (LD.nleaf == 0) continue;
    const Level& L = P.L(ell);
    const int64_t npts = (int64_t)L.sp * L.sp * L.sp;
    if (!LD.gptr_r) {
      LD.gptr_r = M.alloc<int32_t>(LD.nleaf * (npts + 1));
      LD.gptr_t = M.alloc<int32_t>(LD.nleaf * (npts + 1));
    }
    launch_gather_build<R>(F.mr, h->mr_base, h->mr_ext, h->mr_off, F.mt, h->mt_base, h->mt_ext, h->mt_off,
                           h->d_box_rwg_ptr + LD.leaf0, h->d_sc_box_ptr + LD.leaf0, LD.nleaf, L.sp, LD.gptr_r,
                           LD.gptr_t, F.gr, F.gt, s);
    cuda_check(cudaGetLastError(), "gather lists");
  }
  F.lv.assign(P.lv.size(), {});
  for (int ell = P.D; ell >= P.top; --ell) {
    Level& L = P.L(ell);
    auto& FL = F.lv[ell - P.top];
    std::vector<cpx_t<R>> mf(L.Mf.size()), mb(L.Mb.size());
    for (size_t i = 0; i < mf.size(); ++i) mf[i] = mk<R>((R)L.Mf[i].real(), (R)L.Mf[i].imag());
    for (size_t i = 0; i < mb.size(); ++i) mb[i] = mk<R>((R)L.Mb[i].real(), (R)L.Mb[i].imag());
    FL.Mf = M.upload(mf);
    FL.Mb = M.upload(mb);
    if (ell > P.top) {
      const Level& U = P.L(ell - 1);
      int sp = L.sp, spp = U.sp;
      std::vector<R> cl(L.CL.begin(), L.CL.end()), cr(L.CR.begin(), L.CR.end());
      std::vector<R> clt((size_t)sp * spp), crt((size_t)sp * spp);
      for (int j = 0; j < spp; ++j)
        for (int i = 0; i < sp; ++i) {
          clt[(size_t)i * spp + j] = (R)L.CL[(size_t)j * sp + i];
          crt[(size_t)i * spp + j] = (R)L.CR[(size_t)j * sp + i];
        }
      FL.CL = M.upload(cl);
      FL.CR = M.upload(cr);
      FL.CLt = M.upload(clt);
      FL.CRt = M.upload(crt);
    }
  }
  F.built = true;
}

// kernel spectra K^_o for every level (FP64), converted to R
template <typename R>
void build_spectra(efie_handle* h, FarSet<R>& F, const std::vector<double2*>& K64, cudaStream_t s,
                   int comp = -1) {
  Plan& P = h->plan;
  for (int ell = P.D; ell >= P.top; --ell) {
    const LevDev& LD = h->lev[ell - P.top];
    const Level& L = P.L(ell);
    int64_t n3 = (int64_t)L.nfft * L.nfft * L.nfft;
    int64_t tot = n3 * std::max<int64_t>(LD.O, 1);
    cpx_t<R>*& dst = comp < 0 ? F.lv[ell - P.top].Kh : F.lv[ell - P.top].KH[comp];
    if (sizeof(R) == 8) {
      dst = (cpx_t<R>*)K64[ell - P.top];
    } else {
      dst = h->mem.alloc<cpx_t<R>>(tot);
      launch_convert<R>(K64[ell - P.top], dst, LD.O * n3, s);
    }
  }
}

std::vector<double2*> build_kernel_spectra64(efie_handle* h, cudaStream_t s, int comp = -1) {
  Plan& P = h->plan;
  std::vector<double2*> out(P.lv.size(), nullptr);
  for (int ell = P.D; ell >= P.top; --ell) {
    const LevDev& LD = h->lev[ell - P.top];
    const Level& L = P.L(ell);
    const int n = L.nfft;
    const int64_t n3 = (int64_t)n * n * n;
    const int64_t O = LD.O;
    double2* Kh = h->mem.alloc<double2>(n3 * std::max<int64_t>(O, 1));
    out[ell - P.top] = Kh;
    if (O == 0) continue;
    double2* Fn = h->mem.alloc<double2>((int64_t)n * n);
    std::vector<double2> fh((size_t)n * n);
    for (size_t i = 0; i < fh.size(); ++i) fh[i] = make_double2(L.Fn[i].real(), L.Fn[i].imag());
    cuda_check(cudaMemcpy(Fn, fh.data(), sizeof(double2) * fh.size(), cudaMemcpyHostToDevice), "Fn");
    // offsets per pass: two work buffers of <= 512 MiB each, less when a
    // device_mem_limit leaves less room
    int64_t room = (int64_t)(512LL << 20);
    if (h->mem.limit > 0) room = std::min(room, (h->mem.limit - h->mem.bytes - (int64_t)n * n * 16) / 2);
    int64_t ob = std::max<int64_t>(1, std::min<int64_t>(O, room / (n3 * 16)));
    double2* a = h->mem.alloc<double2>(ob * n3);
    double2* b = h->mem.alloc<double2>(ob * n3);
    for (int64_t o0 = 0; o0 < O; o0 += ob) {
      int64_t no = std::min(ob, O - o0);
      launch_kernel_samples(a, LD.offsets, o0, no, n, L.shat, L.h, L.Delta, P.k, comp, s);
      // [o][i0][i1][i2] -> DFT along each axis; last pass writes frequency-major
      View v0{n3, (int64_t)n * n, n, 1};
      launch_mode<double>(a, v0, b, v0, no, 1, 0, n, n, n, n, Fn, Fn, true, nullptr, nullptr, false, s);
      launch_mode<double>(b, v0, a, v0, no, 1, 1, n, n, n, n, Fn, Fn, true, nullptr, nullptr, false, s);
      View vf{1, (int64_t)n * n * O, (int64_t)n * O, O};
      launch_mode<double>(a, v0, Kh + o0, vf, no, 1, 2, n, n, n, n, Fn, Fn, true, nullptr, nullptr, false, s);
    }
    cuda_check(cudaStreamSynchronize(s), "kernel spectra");
    h->mem.release(a);
    h->mem.release(b);
    h->mem.release(Fn);
  }
  return out;
}

template <typename R>
void ensure_far_buffers(efie_handle* h, FarSet<R>& F, int Rc) {
  if (F.Rc >= Rc) return;
  Plan& P = h->plan;
  for (auto* p : F.q) h->mem.release(p);
  for (auto* p : F.r) h->mem.release(p);
  for (void* p : {(void*)F.tmp1, (void*)F.tmp2, (void*)F.Qh, (void*)F.Rh})
    if (p) h->mem.release(p);
  const int64_t C = 4 * Rc;
  F.q.assign(P.lv.size(), nullptr);
  F.r.assign(P.lv.size(), nullptr);
  int64_t tmax = 1, smax = 1;
  for (int ell = P.D; ell >= P.top; --ell) {
    const Level& L = P.L(ell);
    const int64_t B = (int64_t)L.code.size();
    const int64_t sp = L.sp, n = L.nfft;
    F.q[ell - P.top] = h->mem.alloc<cpx_t<R>>(B * sp * sp * sp * C);
    F.r[ell - P.top] = h->mem.alloc<cpx_t<R>>(B * sp * sp * sp * C);
    // forward / inverse intermediates
    tmax = std::max({tmax, B * n * sp * sp * C, B * n * n * sp * C, B * sp * n * n * C});
    smax = std::max(smax, B * n * n * n * C);
    if (ell > P.top) {
      // upward and downward intermediates (child level ell, parent ell-1)
      const int64_t spp = P.L(ell - 1).sp;
      tmax = std::max({tmax, B * spp * sp * sp * C, B * spp * spp * sp * C, B * spp * spp * spp * C,
                       B * sp * spp * spp * C, B * sp * sp * spp * C});
    }
  }
  F.tmp1 = h->mem.alloc<cpx_t<R>>(tmax);
  F.tmp2 = h->mem.alloc<cpx_t<R>>(tmax);
  F.Qh = h->mem.alloc<cpx_t<R>>(smax);
  F.Rh = h->mem.alloc<cpx_t<R>>(smax);
  F.Rc = Rc;
}

void ensure_work(efie_handle* h, int Rw) {
  if (h->Rw >= Rw) return;
  for (void* p : {(void*)h->xs, (void*)h->yA, (void*)h->rho, (void*)h->w, (void*)h->xs4, (void*)h->rho4,
                  (void*)h->xsf, (void*)h->rhof, (void*)h->yAn, (void*)h->wn, (void*)h->wd})
    h->mem.release(p);
  const int64_t N = h->plan.g.N, Nt = h->plan.g.nt;
  h->xs = h->mem.alloc<double2>(N * Rw);
  h->yA = h->mem.alloc<double2>(N * Rw);
  h->rho = h->mem.alloc<double2>(Nt * Rw);
  h->w = h->mem.alloc<double2>(h->n_sc * Rw);
  h->yAn = h->mem.alloc<double2>(N * Rw);
  h->wn = h->mem.alloc<double2>(h->n_sc * Rw);
  if (h->dyadic) h->wd = h->mem.alloc<double2>(h->n_sc * Rw);
  if (h->near_df) {
    h->xs4 = h->mem.alloc<float4>(N * Rw);
    h->rho4 = h->mem.alloc<float4>(Nt * Rw);
  }
  if (h->precision == EFIE_MIXED) {
    h->xsf = h->mem.alloc<float2>(N * Rw);
    h->rhof = h->mem.alloc<float2>(Nt * Rw);
  }
  h->Rw = Rw;
}

// buffers of the second chunk of a pair (FP32 far field, 8 right-hand sides):
// its level grids q2[], r2[], and spectra buffers of the size of the largest
// level (Qt2 for its sources, Rt2 for its results)
void ensure_pair_buffers(efie_handle* h, FarSet<float>& F) {
  if (F.Qt2) return;
  Plan& P = h->plan;
  const int64_t C = 32;
  F.q2.assign(P.lv.size(), nullptr);
  F.r2.assign(P.lv.size(), nullptr);
  for (int ell = P.D; ell >= P.top; --ell) {
    const Level& L = P.L(ell);
    const int64_t sp = L.sp;
    F.q2[ell - P.top] = h->mem.alloc<float2>((int64_t)L.code.size() * sp * sp * sp * C);
    F.r2[ell - P.top] = h->mem.alloc<float2>((int64_t)L.code.size() * sp * sp * sp * C);
  }
  int64_t smax = 1;
  for (int ell = P.D; ell >= P.top; --ell) {
    const Level& L = P.L(ell);
    const int64_t n = L.nfft;
    smax = std::max(smax, (int64_t)L.code.size() * n * n * n * C);
  }
  F.Qt2 = h->mem.alloc<float2>(smax);
  F.Rt2 = h->mem.alloc<float2>(smax);
}

// ------------------------------------------------------------- far pipeline
// The far pipeline of one chunk of nr <= 8 right-hand sides (work-vector
// slots rhs0 .. rhs0 + nr - 1) in pieces, so that two chunks can share the
// translation pass of every level:
//   anterp_up:   anterpolation into the leaf grids and upward transfers (qq[]);
//   fwd_level:   stabilized forward transform of one level (grids -> spectra);
//   run_mac:     translation of one level (spectra -> spectra);
//   inv_level:   inverse transform of one level (spectra -> grids rr[]);
//   down_interp: downward transfers and interpolation.
template <typename R>
void run_mac(efie_handle* h, FarSet<R>& F, int ell, int C, const cpx_t<R>* Qin, cpx_t<R>* Rout, cudaStream_t s);
template <typename R>
void down_interp(efie_handle* h, FarSet<R>& F, int nr, int rhs0, std::vector<cpx_t<R>*>& rr, cudaStream_t s,
                 double2* yout = nullptr, double2* wout = nullptr);

template <typename R>
void anterp_up(efie_handle* h, FarSet<R>& F, int nr, int rhs0, std::vector<cpx_t<R>*>& qq, cudaStream_t s) {
  Plan& P = h->plan;
  const int C = 4 * nr;
  const int D = P.D, top = P.top;
  const int64_t N = P.g.N, Nt = P.g.nt;
  // anterpolation of the currents and charges into the grids of the leaves
  // of level ell (Sec. VI-A; every box of level D in a uniform tree)
  auto anterp = [&](int ell) {
    const Level& L = P.L(ell);
    const LevDev& LV = h->lev[ell - top];
    if (LV.nleaf == 0) return;
    const cpx_t<R>* xin = (const cpx_t<R>*)(h->xs + (int64_t)rhs0 * N);
    // scalar part: the charges (star) or the currents themselves (direct)
    const cpx_t<R>* rin = h->direct ? xin : (const cpx_t<R>*)(h->rho + (int64_t)rhs0 * Nt);
    KScope ks(h, K_ANTERP, s, sizeof(R) == 4 ? (h->direct ? 2 : 3) : 1);
    if (sizeof(R) == 4) {
      launch_convert<R>(h->xs + (int64_t)rhs0 * N, (cpx_t<R>*)(h->xsf + (int64_t)rhs0 * N), N * nr, s);
      if (!h->direct)
        launch_convert<R>(h->rho + (int64_t)rhs0 * Nt, (cpx_t<R>*)(h->rhof + (int64_t)rhs0 * Nt), Nt * nr, s);
      xin = (const cpx_t<R>*)(h->xsf + (int64_t)rhs0 * N);
      rin = h->direct ? xin : (const cpx_t<R>*)(h->rhof + (int64_t)rhs0 * Nt);
    }
    launch_anterp<R>(F.gr, F.gt, LV.gptr_r, LV.gptr_t, h->mr_off, h->mt_off, h->d_box_rwg_ptr + LV.leaf0,
                     h->d_sc_box_ptr + LV.leaf0, LV.nleaf, LV.leaf_box, xin, N, rin, h->direct ? N : Nt, nr,
                     qq[ell - top], L.sp, s);
  };
  anterp(D);
  // upward transfers (Sec. IV-B), shared among siblings one axis at a time (z,
  // y, x); a nonuniform tree's leaves on the parent level are anterpolated
  // after the transfer into that level, over its zeros
  for (int ell = D; ell > top; --ell) {
    KScope ks(h, K_UP, s, 3);
    const Level& L = P.L(ell);
    const Level& U = P.L(ell - 1);
    const LevDev& LD = h->lev[ell - top];
    auto& FL = F.lv[ell - top];
    const int64_t Bp = (int64_t)U.code.size();
    const int sp = L.sp, spp = U.sp;
    View vq{(int64_t)sp * sp * sp * C, (int64_t)sp * sp * C, (int64_t)sp * C, C};
    View t1{(int64_t)sp * sp * spp * C, (int64_t)sp * spp * C, (int64_t)spp * C, C};
    View t2{(int64_t)sp * spp * spp * C, (int64_t)spp * spp * C, (int64_t)spp * C, C};
    View vp{(int64_t)spp * spp * spp * C, (int64_t)spp * spp * C, (int64_t)spp * C, C};
    launch_mode_pair<R>(qq[ell - top], vq, F.tmp1, t1, LD.ng1, C, 2, sp, sp, sp, spp, FL.CL, FL.CR, LD.uz_s0,
                        LD.uz_s1, LD.uz_b0, LD.uz_b1, s);
    launch_mode_pair<R>(F.tmp1, t1, F.tmp2, t2, LD.ng2, C, 1, sp, sp, spp, spp, FL.CL, FL.CR, LD.uy_s0,
                        LD.uy_s1, LD.uy_b0, LD.uy_b1, s);
    launch_mode_pair<R>(F.tmp2, t2, qq[ell - 1 - top], vp, Bp, C, 0, sp, spp, spp, spp, FL.CL, FL.CR, LD.ux_s0,
                        LD.ux_s1, LD.ux_b0, LD.ux_b1, s);
    anterp(ell - 1);
  }
}

template <typename R>
void fwd_level(efie_handle* h, FarSet<R>& F, int ell, int C, const cpx_t<R>* qin, cpx_t<R>* Qout, cudaStream_t s) {
  Plan& P = h->plan;
  const Level& L = P.L(ell);
  auto& FL = F.lv[ell - P.top];
  const int64_t B = (int64_t)L.code.size();
  const int sp = L.sp, n = L.nfft;
  View vq{(int64_t)sp * sp * sp * C, (int64_t)sp * sp * C, (int64_t)sp * C, C};
  View a1{(int64_t)n * sp * sp * C, (int64_t)sp * sp * C, (int64_t)sp * C, C};
  View a2{(int64_t)n * n * sp * C, (int64_t)n * sp * C, (int64_t)sp * C, C};
  View vf{C, (int64_t)n * n * B * C, (int64_t)n * B * C, B * C};
  // y and z passes fused per (box, x-frequency) slab, no y-pass intermediate in HBM
  const bool fuse = sizeof(R) == 4 && C == 32 &&
                    (h->fft_variant == 1 || h->fft_variant == 2 || (h->fft_variant == 3 && sp == 9)) &&
                    dft_yz_fits(sp, n);
  KScope ks(h, K_FWD, s, fuse ? 2 : 3);
  if (!launch_dft<R>(qin, vq, F.tmp1, a1, B, C, 0, sp, n, sp, sp, FL.Mf, n, false, s))
    launch_mode<R>(qin, vq, F.tmp1, a1, B, C, 0, sp, n, sp, sp, FL.Mf, FL.Mf, true, nullptr, nullptr, false, s);
  if (fuse &&
      launch_dft_yz(reinterpret_cast<const float2*>(F.tmp1), reinterpret_cast<float2*>(Qout), B, sp, n,
                    reinterpret_cast<const float2*>(FL.Mf), false, s))
    return;
  if (!launch_dft<R>(F.tmp1, a1, F.tmp2, a2, B, C, 1, sp, n, n, sp, FL.Mf, n, false, s))
    launch_mode<R>(F.tmp1, a1, F.tmp2, a2, B, C, 1, sp, n, n, sp, FL.Mf, FL.Mf, true, nullptr, nullptr, false, s);
  if (!launch_dft<R>(F.tmp2, a2, Qout, vf, B, C, 2, sp, n, n, n, FL.Mf, n, false, s))
    launch_mode<R>(F.tmp2, a2, Qout, vf, B, C, 2, sp, n, n, n, FL.Mf, FL.Mf, true, nullptr, nullptr, false, s);
}

template <typename R>
void inv_level(efie_handle* h, FarSet<R>& F, int ell, int C, const cpx_t<R>* Rin, cpx_t<R>* rout, cudaStream_t s) {
  Plan& P = h->plan;
  const Level& L = P.L(ell);
  auto& FL = F.lv[ell - P.top];
  const int64_t B = (int64_t)L.code.size();
  const int sp = L.sp, n = L.nfft;
  View vq{(int64_t)sp * sp * sp * C, (int64_t)sp * sp * C, (int64_t)sp * C, C};
  View vf{C, (int64_t)n * n * B * C, (int64_t)n * B * C, B * C};
  View b1{(int64_t)sp * n * n * C, (int64_t)n * n * C, (int64_t)n * C, C};
  View b2{(int64_t)sp * sp * n * C, (int64_t)sp * n * C, (int64_t)n * C, C};
  // z and y passes fused per (box, x-frequency) slab into t[b][fx][y][z][c], then the x pass
  const bool fuse = sizeof(R) == 4 && C == 32 && (h->fft_variant == 2 || (h->fft_variant == 3 && sp == 9)) &&
                    dft_zy_fits(sp, n);
  KScope ks(h, K_INV, s, fuse ? 2 : 3);
  if (fuse &&
      launch_dft_yz(reinterpret_cast<const float2*>(Rin), reinterpret_cast<float2*>(F.tmp1), B, sp, n,
                    reinterpret_cast<const float2*>(FL.Mb), true, s)) {
    View vt{(int64_t)n * sp * sp * C, (int64_t)sp * sp * C, (int64_t)sp * C, C};
    if (!launch_dft<R>(F.tmp1, vt, rout, vq, B, C, 0, n, sp, sp, sp, FL.Mb, n, true, s))
      launch_mode<R>(F.tmp1, vt, rout, vq, B, C, 0, n, sp, sp, sp, FL.Mb, FL.Mb, true, nullptr, nullptr, false, s);
    return;
  }
  if (!launch_dft<R>(Rin, vf, F.tmp1, b1, B, C, 0, n, sp, n, n, FL.Mb, n, true, s))
    launch_mode<R>(Rin, vf, F.tmp1, b1, B, C, 0, n, sp, n, n, FL.Mb, FL.Mb, true, nullptr, nullptr, false, s);
  if (!launch_dft<R>(F.tmp1, b1, F.tmp2, b2, B, C, 1, n, sp, sp, n, FL.Mb, n, true, s))
    launch_mode<R>(F.tmp1, b1, F.tmp2, b2, B, C, 1, n, sp, sp, n, FL.Mb, FL.Mb, true, nullptr, nullptr, false, s);
  if (!launch_dft<R>(F.tmp2, b2, rout, vq, B, C, 2, n, sp, sp, sp, FL.Mb, n, true, s))
    launch_mode<R>(F.tmp2, b2, rout, vq, B, C, 2, n, sp, sp, sp, FL.Mb, FL.Mb, true, nullptr, nullptr, false, s);
}

// grids and spectra of the Hessian translation (dyadic factorization) for
// chunks of up to Rc right-hand sides
template <typename R>
void ensure_dyad_buffers(efie_handle* h, FarSet<R>& F, int Rc) {
  if (F.Rd >= Rc) return;
  Plan& P = h->plan;
  for (auto* p : F.rd) h->mem.release(p);
  if (F.Rdh) h->mem.release(F.Rdh);
  const int64_t C = 4 * Rc;
  F.rd.assign(P.lv.size(), nullptr);
  int64_t smax = 1;
  for (int ell = P.D; ell >= P.top; --ell) {
    const Level& L = P.L(ell);
    const int64_t B = (int64_t)L.code.size(), sp = L.sp, n = L.nfft;
    F.rd[ell - P.top] = h->mem.alloc<cpx_t<R>>(B * sp * sp * sp * C);
    smax = std::max(smax, B * n * n * n * C);
  }
  F.Rdh = h->mem.alloc<cpx_t<R>>(smax);
  F.Rd = Rc;
}

template <typename R>
void far_chunk(efie_handle* h, FarSet<R>& F, int nr, cudaStream_t s) {
  Plan& P = h->plan;
  const int C = 4 * nr;
  if (h->dyadic) ensure_dyad_buffers<R>(h, F, nr);
  anterp_up<R>(h, F, nr, 0, F.q, s);
  for (int ell = P.D; ell >= P.top; --ell) {
    const Level& L = P.L(ell);
    const int64_t sp = L.sp;
    if (h->lev[ell - P.top].nfar == 0) {
      const size_t bytes = sizeof(cpx_t<R>) * (int64_t)L.code.size() * sp * sp * sp * C;
      cuda_check(cudaMemsetAsync(F.r[ell - P.top], 0, bytes, s), "memset r");
      if (h->dyadic) cuda_check(cudaMemsetAsync(F.rd[ell - P.top], 0, bytes, s), "memset r");
      continue;
    }
    fwd_level<R>(h, F, ell, C, F.q[ell - P.top], F.Qh, s);
    run_mac<R>(h, F, ell, C, F.Qh, F.Rh, s);
    inv_level<R>(h, F, ell, C, F.Rh, F.r[ell - P.top], s);
    if (h->dyadic) {
      // Hessian translation of the same spectra (Sec. VI-C)
      const Level& Lv = P.L(ell);
      const LevDev& LD = h->lev[ell - P.top];
      const auto& FL = F.lv[ell - P.top];
      KH6<R> K;
      for (int c = 0; c < 6; ++c) K.k[c] = FL.KH[c];
      {
        KScope ks(h, K_MAC, s, 1);
        launch_mac_dyad<R>(F.Qh, F.Rdh, K, (int64_t)Lv.code.size(), nr, (int64_t)Lv.nfft * Lv.nfft * Lv.nfft, LD.O,
                           LD.il_ptr, LD.il_src, LD.il_off, s);
      }
      inv_level<R>(h, F, ell, C, F.Rdh, F.rd[ell - P.top], s);
    }
  }
  down_interp<R>(h, F, nr, 0, F.r, s);
  if (h->dyadic) {
    // the Hessian grids' vector part is the scalar part of the product, with
    // the sign of int int f_m . grad grad g . f_n = -Phi_mn: w = -(m . r_H)
    down_interp<R>(h, F, nr, 0, F.rd, s, h->w, h->wd);
    KScope ks(h, K_VEC, s, 1);
    launch_lincomb(h->w, h->w, 0.0, -1.0, h->w, h->n_sc * nr, s);
  }
}

template <typename R>
void run_mac(efie_handle* h, FarSet<R>& F, int ell, int C, const cpx_t<R>* Qin, cpx_t<R>* Rout, cudaStream_t s) {
  Plan& P = h->plan;
  const int top = P.top;
  const Level& L = P.L(ell);
  const LevDev& LD = h->lev[ell - top];
  auto& FL = F.lv[ell - top];
  const int64_t B = (int64_t)L.code.size();
  const int n = L.nfft;
  const int64_t n3 = (int64_t)n * n * n;
    {
      const bool autov = h->mac_variant == 0 || h->mac_variant == 4;
      const bool tc3 = sizeof(R) == 4 && h->mac_variant == 5 &&
                       mac_top_tc3_fits(C, LD.max_tile, LD.O, LD.nq, LD.ntiles, 1);
      const bool tc2 = sizeof(R) == 4 && (autov || h->mac_variant == 5) && !tc3 && LD.tile_k16 &&
                       mac_top_tc2_fits(C, LD.max_tile, LD.O, LD.nq, LD.ntiles, 1);
      const bool tc = sizeof(R) == 4 && (autov || h->mac_variant == 3) &&
                      mac_top_tc_fits(C, LD.max_tile, LD.O);
      KScope ks(h, tc || tc2 || tc3 ? K_MAC_TOP_TC : ell == top ? K_MAC_TOP : K_MAC, s, 1);
      bool done = false;
      if (tc3 || tc2) {
        const float2* qv[1] = {(const float2*)Qin};
        float2* rv[1] = {(float2*)Rout};
        done = tc3 ? launch_mac_top_tc3(qv, rv, 1, (const float2*)FL.Kh, B, C, LD.O, n3, LD.ntiles, LD.max_tile,
                                        LD.tile_tgt_ptr, LD.tile_tgt, LD.tile_src_ptr, LD.tile_src,
                                        LD.tile_kidx_off, LD.tile_kidx, LD.nq, h->err_dev, s)
                   : launch_mac_top_tc2(qv, rv, 1, (const float2*)FL.Kh, B, C, LD.O, n3, LD.ntiles, LD.max_tile,
                                        LD.tile_tgt_ptr, LD.tile_tgt, LD.tile_src_ptr, LD.tile_src,
                                        LD.tile_k16_off, LD.tile_k16, LD.nq, h->err_dev, s);
      }
      if (done) cuda_check(cudaPeekAtLastError(), "top-level translation (persistent tensor-core kernel)");
      if (!done && tc)
        done = launch_mac_top_tc((const float2*)Qin, (float2*)Rout, (const float2*)FL.Kh, B, C, LD.O, n3,
                                 LD.ntiles, LD.max_tile, LD.tile_tgt_ptr, LD.tile_tgt, LD.tile_src_ptr, LD.tile_src,
                                 LD.tile_kidx_off, LD.tile_kidx, h->err_dev, s);
      if (done) cuda_check(cudaPeekAtLastError(), "top-level translation (tensor-core kernel)");
      if (!done)
        launch_mac<R>(Qin, Rout, FL.Kh, B, C, LD.O, n3, LD.ntiles,
                      h->mac_variant == 1 ? -LD.max_tile : LD.max_tile, LD.tile_tgt_ptr, LD.tile_tgt,
                      LD.tile_src_ptr, LD.tile_src, LD.tile_kidx_off, LD.tile_kidx, s);
    }
}

// downward transfers and interpolation of the output grids rr into the
// vector part yout (default h->yA) and the scalar part wout (default h->w)
template <typename R>
void down_interp(efie_handle* h, FarSet<R>& F, int nr, int rhs0, std::vector<cpx_t<R>*>& rr, cudaStream_t s,
                 double2* yout, double2* wout) {
  Plan& P = h->plan;
  const int C = 4 * nr;
  const int D = P.D, top = P.top;
  const int64_t N = P.g.N, Nt = P.g.nt;
  // downward transfers r_c += C^T r_parent (Sec. IV-B), shared among siblings one
  // axis at a time (x for (parent, b_x), y for (parent, b_x, b_y), z per child)
  for (int ell = top + 1; ell <= D; ++ell) {
    KScope ks(h, K_DOWN, s, 3);
    const Level& L = P.L(ell);
    const Level& U = P.L(ell - 1);
    const LevDev& LD = h->lev[ell - top];
    auto& FL = F.lv[ell - top];
    int64_t B = (int64_t)L.code.size();
    int sp = L.sp, spp = U.sp;
    View vp{(int64_t)spp * spp * spp * C, (int64_t)spp * spp * C, (int64_t)spp * C, C};
    View w1{(int64_t)sp * spp * spp * C, (int64_t)spp * spp * C, (int64_t)spp * C, C};
    View w2{(int64_t)sp * sp * spp * C, (int64_t)sp * spp * C, (int64_t)spp * C, C};
    View vq{(int64_t)sp * sp * sp * C, (int64_t)sp * sp * C, (int64_t)sp * C, C};
    launch_mode<R>(rr[ell - 1 - top], vp, F.tmp1, w1, LD.ng2, C, 0, spp, sp, spp, spp, FL.CLt, FL.CRt, false,
                   LD.dx_sel, LD.dx_src, false, s);
    launch_mode<R>(F.tmp1, w1, F.tmp2, w2, LD.ng1, C, 1, spp, sp, sp, spp, FL.CLt, FL.CRt, false, LD.dy_sel,
                   LD.dy_src, false, s);
    launch_mode<R>(F.tmp2, w2, rr[ell - top], vq, B, C, 2, spp, sp, sp, sp, FL.CLt, FL.CRt, false, LD.bits,
                   LD.dz_src, true, s);
  }
  // interpolation onto the RWG test functions and the charges (Sec. VI-A),
  // level by level over the functions whose leaves lie there
  double2* ya = (yout ? yout : h->yA) + (int64_t)rhs0 * N;
  double2* wa = (wout ? wout : h->w) + (int64_t)rhs0 * h->n_sc;
  const int64_t* sc_ptr = h->direct ? P.box_rwg_ptr.data() : P.box_tri_ptr.data();
  for (int ell = top; ell <= D; ++ell) {
    const LevDev& LV = h->lev[ell - top];
    if (LV.nleaf == 0) continue;
    KScope ks(h, K_INTERP, s, 1);
    const Level& L = P.L(ell);
    const int64_t i0 = P.box_rwg_ptr[LV.leaf0], i1 = P.box_rwg_ptr[LV.leaf0 + LV.nleaf];
    const int64_t t0 = sc_ptr[LV.leaf0], t1 = sc_ptr[LV.leaf0 + LV.nleaf];
    launch_interp<R>(F.mr, h->mr_base + 3 * i0, h->mr_ext + 3 * i0, h->mr_off + i0, h->d_rwg_lbox + i0, i1 - i0,
                     F.mt, h->mt_base + 3 * t0, h->mt_ext + 3 * t0, h->mt_off + t0, h->d_sc_lbox + t0, t1 - t0,
                     rr[ell - top], L.sp, nr, ya + i0, N, wa + t0, h->n_sc, s);
  }
}



// the near field (Sec. VI-A; FP64 class) of nr right-hand sides into yAn / wn, on
// the handle's second stream, after the charges on `s` (fork); the far field
// runs meanwhile on `s`.  near_join makes `s` wait for it, and combine adds
// the near and far parts.
void near_fork(efie_handle* h, int nr, cudaStream_t s) {
  Plan& P = h->plan;
  const int64_t N = P.g.N, Nt = P.g.nt;
  const int64_t BD = P.n_leaves;
  cudaStream_t sn = h->s_near;
  cuda_check(cudaEventRecord(h->ev_fork, s), "near fork");
  cuda_check(cudaStreamWaitEvent(sn, h->ev_fork, 0), "near fork");
  cuda_check(cudaStreamWaitEvent(h->s_far, h->ev_fork, 0), "far fork");
  cuda_check(cudaMemsetAsync(h->yAn, 0, sizeof(double2) * N * nr, sn), "near outputs");
  cuda_check(cudaMemsetAsync(h->wn, 0, sizeof(double2) * h->n_sc * nr, sn), "near outputs");
  if (h->near_df) {
    {
      KScope ks(h, K_NEAR_A, sn, 2);
      launch_split_vec(h->xs, h->xs4, N * nr, sn);
      launch_near_spmv_df((const float4*)h->nd.A, h->d_blkA_off, h->d_near_ptr, h->d_near_src, h->d_box_rwg_ptr,
                          BD, h->xs4, h->yAn, N, nr, h->near_variant, h->err_dev, sn);
    }
    {
      KScope ks(h, K_NEAR_V, sn, 2);
      // scalar part: V on the charges (star), or Phi on the currents (direct)
      if (!h->direct) launch_split_vec(h->rho, h->rho4, Nt * nr, sn);
      launch_near_spmv_df((const float4*)h->nd.Vn, h->d_blkS_off, h->d_near_ptr, h->d_near_src, h->d_sc_box_ptr,
                          BD, h->direct ? h->xs4 : h->rho4, h->wn, h->n_sc, nr, h->near_variant, h->err_dev, sn);
    }
  } else {
    {
      KScope ks(h, K_NEAR_A, sn, 1);
      launch_near_spmv(h->nd.A, h->d_blkA_off, h->d_near_ptr, h->d_near_src, h->d_box_rwg_ptr, BD, h->xs,
                       h->yAn, N, nr, sn);
    }
    {
      KScope ks(h, K_NEAR_V, sn, 1);
      launch_near_spmv(h->nd.Vn, h->d_blkS_off, h->d_near_ptr, h->d_near_src, h->d_sc_box_ptr, BD,
                       h->direct ? h->xs : h->rho, h->wn, h->n_sc, nr, sn);
    }
  }
  cuda_check(cudaEventRecord(h->ev_join, sn), "near join");
  // while kernel classes are being timed, the far field waits for the near
  // field, so that no class's events include another class running beside it
  if (h->prof.on) cuda_check(cudaStreamWaitEvent(h->s_far, h->ev_join, 0), "near join");
}

void near_join_combine(efie_handle* h, int nr, double2* y, double2* yAo, double2* yVo, int64_t ldy, cudaStream_t s) {
  Plan& P = h->plan;
  const int64_t N = P.g.N, Nt = P.g.nt;
  cuda_check(cudaEventRecord(h->ev_far, h->s_far), "far join");
  cuda_check(cudaStreamWaitEvent(s, h->ev_far, 0), "far join");
  cuda_check(cudaStreamWaitEvent(s, h->ev_join, 0), "near join");
  std::complex<double> cA = jk_of(P.k), cV = 1.0 / jk_of(P.k);
  KScope ks(h, K_VEC, s, 1);
  launch_combine(h->yA, N, h->w, h->n_sc, h->yAn, h->wn, h->d_rwg_perm, h->direct ? nullptr : h->d_rwg_tri_sorted,
                 N, nr,
                 make_double2(cA.real(), cA.imag()), make_double2(cV.real(), cV.imag()), y, ldy, yAo, yVo,
                 s);
}

// y = T x (or parts) for nr <= 8 right-hand sides; x, y canonical [nr][ldx]
template <typename R>
void matvec_chunk(efie_handle* h, FarSet<R>& F, const double2* x, int64_t ldx, int nr, double2* y,
                  double2* yAo, double2* yVo, int64_t ldy, cudaStream_t s) {
  Plan& P = h->plan;
  const int64_t N = P.g.N, Nt = P.g.nt;
  ensure_work(h, 8);
  ensure_far_buffers(h, F, nr);
  {
    KScope ks(h, K_VEC, s, h->direct ? 1 : 2);
    launch_permute_in(x, ldx, h->d_rwg_perm, N, nr, h->xs, s);
    if (!h->direct) launch_charges(h->xs, N, h->d_tri_rwg, h->d_tri_sgn, Nt, nr, h->rho, Nt, s);  // rho = Sigma^T x
  }
  near_fork(h, nr, s);                                                             // near field
  far_chunk<R>(h, F, nr, h->s_far);                                                // far field
  near_join_combine(h, nr, y, yAo, yVo, ldy, s);
}

// Whether two full chunks (16 right-hand sides) can share the translation
// passes: FP32 far field, the automatic translation choice, and a top grid
// level that the persistent tensor-core kernel takes with 128-row B operands.
bool pair_fits(efie_handle* h) {
  if (h->precision != EFIE_MIXED || h->dyadic ||
      (h->mac_variant != 0 && h->mac_variant != 4 && h->mac_variant != 5))
    return false;
  const LevDev& LD = h->lev[0];
  return LD.nfar > 0 && (mac_top_tc3_fits(32, LD.max_tile, LD.O, LD.nq, LD.ntiles, 2) ||
                         (LD.tile_k16 && mac_top_tc2_fits(32, LD.max_tile, LD.O, LD.nq, LD.ntiles, 2)));
}

// The translation of level ell for both chunks of a pair (spectra Qa, Qb ->
// Ra, Rb): one tensor-core pass over 64 channels with the level's 128-target
// tiles (the top level's own tiles, or the interaction-list tiles below it),
// or one pass per chunk on the single-chunk kernels when those do not fit.
void run_mac_pair(efie_handle* h, int ell, const float2* Qa, const float2* Qb, float2* Ra, float2* Rb,
                  cudaStream_t s) {
  Plan& P = h->plan;
  FarSet<float>& F = h->f32;
  const Level& L = P.L(ell);
  const LevDev& LD = h->lev[ell - P.top];
  const int64_t n = L.nfft, B = (int64_t)L.code.size();
  const bool top = ell == P.top;
  const int64_t nt = top ? LD.ntiles : LD.tct_ntiles, nq = top ? LD.nq : LD.tct_nq;
  const int mx = top ? LD.max_tile : LD.tct_max;
  const bool il_tc = top || h->mac_variant == 0 || h->mac_variant == 5;
  const bool use3 = h->mac_variant == 5 && nt > 0 && mac_top_tc3_fits(32, mx, LD.O, nq, nt, 2);
  const int16_t* k16 = top ? LD.tile_k16 : LD.tct_k16;
  const bool use2 = !use3 && nt > 0 && k16 && mac_top_tc2_fits(32, mx, LD.O, nq, nt, 2);
  if (il_tc && (use3 || use2)) {
    KScope ks(h, top ? K_MAC_TOP_TC : K_MAC_TC, s, 1);
    const float2* qv[2] = {Qa, Qb};
    float2* rv[2] = {Ra, Rb};
    const float2* Kh = F.lv[ell - P.top].Kh;
    const int64_t nf = n * n * n;
    bool ok;
    if (use3)
      ok = top ? launch_mac_top_tc3(qv, rv, 2, Kh, B, 32, LD.O, nf, nt, mx, LD.tile_tgt_ptr, LD.tile_tgt,
                                    LD.tile_src_ptr, LD.tile_src, LD.tile_kidx_off, LD.tile_kidx, nq, h->err_dev, s)
               : launch_mac_top_tc3(qv, rv, 2, Kh, B, 32, LD.O, nf, nt, mx, LD.tct_tgt_ptr, LD.tct_tgt,
                                    LD.tct_src_ptr, LD.tct_src, LD.tct_kidx_off, LD.tct_kidx, nq, h->err_dev, s);
    else
      ok = top ? launch_mac_top_tc2(qv, rv, 2, Kh, B, 32, LD.O, nf, nt, mx, LD.tile_tgt_ptr, LD.tile_tgt,
                                    LD.tile_src_ptr, LD.tile_src, LD.tile_k16_off, LD.tile_k16, nq, h->err_dev, s)
               : launch_mac_top_tc2(qv, rv, 2, Kh, B, 32, LD.O, nf, nt, mx, LD.tct_tgt_ptr, LD.tct_tgt,
                                    LD.tct_src_ptr, LD.tct_src, LD.tct_k16_off, LD.tct_k16, nq, h->err_dev, s);
    if (!ok) throw EfieError{EFIE_ECUDA, "internal: chunk-pair translation does not apply"};
    cuda_check(cudaPeekAtLastError(), "translation (chunk pair, tensor cores)");
    return;
  }
  run_mac<float>(h, F, ell, 32, Qa, Ra, s);
  run_mac<float>(h, F, ell, 32, Qb, Rb, s);
}

// y = T x for 16 np right-hand sides.  The near field takes all of them in
// one pass over the near matrix on the second stream, while the far field
// runs pair by pair (two chunks of 8): both chunks' upward pipelines, then
// level by level both forward transforms, one translation pass for both,
// both inverse transforms; then each chunk's downward pipeline.
void matvec_pairs(efie_handle* h, const double2* x, int64_t ldx, double2* y, double2* yAo, double2* yVo,
                  int64_t ldy, int np, cudaStream_t s) {
  Plan& P = h->plan;
  FarSet<float>& F = h->f32;
  const int64_t N = P.g.N, Nt = P.g.nt;
  const int R = 16 * np;
  ensure_work(h, R);
  ensure_far_buffers(h, F, 8);
  ensure_pair_buffers(h, F);
  {
    KScope ks(h, K_VEC, s, h->direct ? 1 : 2);
    launch_permute_in(x, ldx, h->d_rwg_perm, N, R, h->xs, s);
    if (!h->direct) launch_charges(h->xs, N, h->d_tri_rwg, h->d_tri_sgn, Nt, R, h->rho, Nt, s);
  }
  near_fork(h, R, s);
  cudaStream_t sf = h->s_far;
  for (int pi = 0; pi < np; ++pi) {
    const int ra = 16 * pi, rb = ra + 8;
    anterp_up<float>(h, F, 8, ra, F.q, sf);
    anterp_up<float>(h, F, 8, rb, F.q2, sf);
    for (int ell = P.D; ell >= P.top; --ell) {
      const Level& L = P.L(ell);
      const int64_t sp = L.sp;
      if (h->lev[ell - P.top].nfar == 0) {
        const size_t bytes = sizeof(float2) * (size_t)L.code.size() * sp * sp * sp * 32;
        cuda_check(cudaMemsetAsync(F.r[ell - P.top], 0, bytes, sf), "memset r");
        cuda_check(cudaMemsetAsync(F.r2[ell - P.top], 0, bytes, sf), "memset r");
        continue;
      }
      fwd_level<float>(h, F, ell, 32, F.q[ell - P.top], F.Qh, sf);
      fwd_level<float>(h, F, ell, 32, F.q2[ell - P.top], F.Qt2, sf);
      run_mac_pair(h, ell, F.Qh, F.Qt2, F.Rh, F.Rt2, sf);
      inv_level<float>(h, F, ell, 32, F.Rh, F.r[ell - P.top], sf);
      inv_level<float>(h, F, ell, 32, F.Rt2, F.r2[ell - P.top], sf);
    }
    down_interp<float>(h, F, 8, ra, F.r, sf);
    down_interp<float>(h, F, 8, rb, F.r2, sf);
  }
  near_join_combine(h, R, y, yAo, yVo, ldy, s);
}

void do_matvec(efie_handle* h, const double2* x, int64_t ldx, double2* y, double2* yA, double2* yV,
               int64_t ldy, int n_rhs, bool force64, cudaStream_t s) {
  // a device wait of an earlier product ran out (its outputs were set to NaN)
  if (h->err_host && *reinterpret_cast<volatile int*>(h->err_host)) {
    *reinterpret_cast<volatile int*>(h->err_host) = 0;
    throw EfieError{EFIE_ETIMEOUT, "a bounded device wait of an earlier product expired"};
  }
  // right-hand sides per far pass: at most 8; the FP64 pass of a mixed handle
  // (true residuals) runs one at a time to bound its buffers
  int Rc = h->opt.rhs_chunk > 0 ? std::min(h->opt.rhs_chunk, 8) : 8;
  if (force64 && h->precision == EFIE_MIXED) Rc = 1;
  Rc = std::min(Rc, n_rhs);
  // full chunk pairs share one top-level tensor-core pass
  const bool pairs = Rc == 8 && !force64 && pair_fits(h);
  for (int r0 = 0; r0 < n_rhs;) {
    double2* yy = y ? y + (int64_t)r0 * ldy : nullptr;
    double2* ya = yA ? yA + (int64_t)r0 * ldy : nullptr;
    double2* yv = yV ? yV + (int64_t)r0 * ldy : nullptr;
    if (pairs && n_rhs - r0 >= 16) {
      // at most 4 pairs (64 right-hand sides) per near-field pass, which
      // bounds the work vectors (they grow with the right-hand sides of a pass)
      const int np = std::min((n_rhs - r0) / 16, 4);
      matvec_pairs(h, x + (int64_t)r0 * ldx, ldx, yy, ya, yv, ldy, np, s);
      r0 += 16 * np;
      continue;
    }
    int nr = std::min(Rc, n_rhs - r0);
    r0 += nr;
    if (h->precision == EFIE_MIXED && !force64)
      matvec_chunk<float>(h, h->f32, x + (int64_t)(r0 - nr) * ldx, ldx, nr, yy, ya, yv, ldy, s);
    else
      matvec_chunk<double>(h, h->f64, x + (int64_t)(r0 - nr) * ldx, ldx, nr, yy, ya, yv, ldy, s);
  }
  cuda_check(cudaGetLastError(), "matvec launch");
}

// ------------------------------------------------------------- setup
// Index tiles (offset ids [source][tpad] per tile, -1 for excluded pairs)
// re-laid out for the persistent tensor-core kernel: per tile, per chunk of
// 16 sources, per target row the 16 ids as int16 (padded with -1), so that a
// producer thread reads its row of a chunk as two 16-byte words.  off[t] is
// the tile's first entry.  Returns false when an id exceeds int16.
bool make_index16(const std::vector<int64_t>& tgt_ptr, const std::vector<int64_t>& src_ptr,
                  const std::vector<int64_t>& kidx_off, const std::vector<int32_t>& kidx,
                  std::vector<int16_t>& out, std::vector<int64_t>& off) {
  const int64_t nt = (int64_t)tgt_ptr.size() - 1;
  off.assign(nt + 1, 0);
  for (int64_t t = 0; t < nt; ++t) {
    const int64_t tpad = ((tgt_ptr[t + 1] - tgt_ptr[t] + 7) / 8) * 8;
    const int64_t nch = (src_ptr[t + 1] - src_ptr[t] + 15) / 16;
    off[t + 1] = off[t] + nch * tpad * 16;
  }
  out.assign(off[nt], (int16_t)-1);
  for (int64_t t = 0; t < nt; ++t) {
    const int64_t tpad = ((tgt_ptr[t + 1] - tgt_ptr[t] + 7) / 8) * 8;
    const int64_t ns = src_ptr[t + 1] - src_ptr[t];
    for (int64_t j = 0; j < ns; ++j)
      for (int64_t r = 0; r < tpad; ++r) {
        const int32_t id = kidx[kidx_off[t] + j * tpad + r];
        if (id > 32767) return false;
        out[off[t] + ((j / 16) * tpad + r) * 16 + (j % 16)] = (int16_t)id;
      }
  }
  return true;
}

// tree: null for the uniform octree of (grid_spacing, levels); else the
// nonuniform octree of Sec. VII with these options (grid_spacing and levels
// unused)
void setup_impl(efie_handle* h, const efie_mesh* mesh, double k, int p, double grid_spacing, int levels,
                const AdaptiveOptions* tree = nullptr) {
  check_mesh(mesh);
  if (h->opt.factorization != EFIE_FACT_STAR && h->opt.factorization != EFIE_FACT_DIRECT &&
      h->opt.factorization != EFIE_FACT_DYADIC)
    throw EfieError{EFIE_EINVAL, "factorization must be EFIE_FACT_STAR, EFIE_FACT_DIRECT or EFIE_FACT_DYADIC"};
  if (tree && h->opt.factorization != EFIE_FACT_STAR)
    throw EfieError{EFIE_EINVAL, "the nonuniform tree takes the star factorization (EFIE_FACT_STAR)"};
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
    throw EfieError{EFIE_ECUDA, "no CUDA device"};
  cuda_check(cudaGetDevice(&h->device), "cudaGetDevice");
  // flag that bounded device waits set when they run out; host-mapped, so the
  // host reads it without synchronising
  cuda_check(cudaHostAlloc((void**)&h->err_host, sizeof(int), cudaHostAllocMapped), "cudaHostAlloc");
  *h->err_host = 0;
  cuda_check(cudaHostGetDevicePointer((void**)&h->err_dev, h->err_host, 0), "cudaHostGetDevicePointer");
  {
    int least = 0, greatest = 0;
    cuda_check(cudaDeviceGetStreamPriorityRange(&least, &greatest), "stream priorities");
    cuda_check(cudaStreamCreateWithPriority(&h->s_near, cudaStreamNonBlocking, least), "near-field stream");
    cuda_check(cudaStreamCreateWithPriority(&h->s_far, cudaStreamNonBlocking, greatest), "far-field stream");
  }
  cuda_check(cudaEventCreateWithFlags(&h->ev_far, cudaEventDisableTiming), "far-field event");
  cuda_check(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming), "near-field event");
  cuda_check(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming), "near-field event");
  h->mem.limit = h->opt.device_mem_limit;
  Plan& P = h->plan;
  using clk = std::chrono::steady_clock;
  auto t_mark = clk::now();
  auto phase_done = [&](int i) {
    const auto now = clk::now();
    h->setup_s[i] = std::chrono::duration<double>(now - t_mark).count();
    t_mark = now;
  };
  h->dyadic = h->opt.factorization == EFIE_FACT_DYADIC;
  h->direct = h->opt.factorization == EFIE_FACT_DIRECT || h->dyadic;
  if (tree)
    build_plan_adaptive(P, mesh->xyz, mesh->n_vertices, mesh->tri, mesh->n_triangles, k, p, *tree, true,
                        h->direct);
  else
    build_plan(P, mesh->xyz, mesh->n_vertices, mesh->tri, mesh->n_triangles, k, p, grid_spacing, levels,
               h->opt.n_splines, true, h->direct);
  // the upward transfer takes at most TRANSFER_MAX_SPLINES splines per axis
  // on every level below the top one: refuse other plans before any device
  // memory is allocated (not at the first product)
  for (int ell = P.top + 1; ell <= P.D; ++ell)
    if (P.L(ell).sp > TRANSFER_MAX_SPLINES)
      throw EfieError{EFIE_EINVAL, "level " + std::to_string(ell) + " has " + std::to_string(P.L(ell).sp) +
                                       " splines per axis; the transfers take at most " +
                                       std::to_string(TRANSFER_MAX_SPLINES) + " below the top level"};
  phase_done(0);
  DevMem& M = h->mem;
  cudaStream_t s = 0;
  // quadrature rules
  {
    std::vector<double> q3, q4, q6;
    collapsed_rule(3, q3);
    collapsed_rule(4, q4);
    collapsed_rule(6, q6);
    if (near_upload_rules(q3.data(), q4.data()) || upload_rhs_rule(q6.data()))
      throw EfieError{EFIE_ECUDA, "constant upload failed"};
  }
  const Geometry& g = P.g;
  const int64_t N = g.N, Nt = g.nt;
  h->dV = M.upload(g.V);
  h->dT = M.upload(g.T);
  h->darea = M.upload(g.area);
  h->dtri_pm = M.upload(g.tri_pm);
  h->dfree_pm = M.upload(g.free_pm);
  h->d_rwg_perm = M.upload(P.rwg_perm);
  h->d_rwg_box = M.upload(P.rwg_box);
  h->d_tri_box = M.upload(P.tri_box);
  h->d_box_rwg_ptr = M.upload(P.box_rwg_ptr);
  h->d_box_tri_ptr = M.upload(P.box_tri_ptr);
  h->d_rwg_tri_sorted = M.upload(P.rwg_tri_sorted);
  h->n_sc = h->direct ? N : Nt;
  h->d_sc_box_ptr = h->direct ? h->d_box_rwg_ptr : h->d_box_tri_ptr;
  h->d_sc_box = h->direct ? h->d_rwg_box : h->d_tri_box;
  h->d_rwg_lbox = P.adaptive ? M.upload(P.rwg_lbox) : h->d_rwg_box;
  h->d_tri_lbox = P.adaptive ? M.upload(P.tri_lbox) : h->d_tri_box;
  h->d_sc_lbox = h->direct ? h->d_rwg_lbox : h->d_tri_lbox;
  {
    // per sorted triangle: its RWGs (sorted index) and signs
    std::vector<int32_t> tr(3 * Nt, -1);
    std::vector<int8_t> ts(3 * Nt, 0);
    std::vector<int> cnt(Nt, 0);
    for (int64_t i = 0; i < N; ++i)
      for (int sd = 0; sd < 2; ++sd) {
        int32_t t = P.rwg_tri_sorted[2 * i + sd];
        if (cnt[t] >= 3) throw EfieError{EFIE_EINVAL, "triangle with more than 3 edges"};
        tr[3 * t + cnt[t]] = (int32_t)i;
        ts[3 * t + cnt[t]] = sd == 0 ? 1 : -1;
        cnt[t]++;
      }
    h->d_tri_rwg = M.upload(tr);
    h->d_tri_sgn = M.upload(ts);
  }
  h->mr_base = M.upload(P.mom_rwg.base);
  h->mr_ext = M.upload(P.mom_rwg.ext);
  h->mr_off = M.upload(P.mom_rwg.off);
  {
    const MomentBlocks& MS = h->direct ? P.mom_div : P.mom_tri;   // scalar-part moments
    h->mt_base = M.upload(MS.base);
    h->mt_ext = M.upload(MS.ext);
    h->mt_off = M.upload(MS.off);
  }
  // levels
  h->lev.assign(P.lv.size(), LevDev());
  for (int ell = P.D; ell >= P.top; --ell) {
    const Level& L = P.L(ell);
    LevDev& LD = h->lev[ell - P.top];
    LD.B = (int64_t)L.code.size();
    LD.leaf0 = P.level_leaf_ptr[ell - P.top];
    LD.nleaf = P.level_leaf_ptr[ell - P.top + 1] - LD.leaf0;
    if (LD.nleaf > 0 && LD.nleaf != LD.B) {
      std::vector<int32_t> lb(LD.nleaf);
      for (int64_t x = 0; x < LD.nleaf; ++x) lb[x] = (int32_t)P.leaf_box[LD.leaf0 + x];
      LD.leaf_box = M.upload(lb);
    }
    LD.il_ptr = M.upload(L.il_ptr);
    LD.il_src = M.upload(L.il_src);
    LD.il_off = M.upload(L.il_off);
    {
      // an even number of kernel spectra per frequency (a copy of the last
      // offset, referenced by no pair), so that every frequency's row of FP32
      // spectra starts on a 16-byte boundary for the bulk copies
      std::vector<int32_t> offs = L.offsets;
      if ((offs.size() / 3) % 2 == 1) offs.insert(offs.end(), L.offsets.end() - 3, L.offsets.end());
      LD.offsets = M.upload(offs);
      LD.O = (int64_t)offs.size() / 3;
    }
    LD.nfar = (int64_t)L.il_src.size();
    LD.parent = M.upload(L.parent);
    std::vector<int8_t> bits(3 * LD.B);
    for (int64_t b = 0; b < LD.B; ++b)
      for (int d = 0; d < 3; ++d) bits[3 * b + d] = (int8_t)(L.ijk[3 * b + d] & 1);
    LD.bits = M.upload(bits);
    if (ell < P.D) LD.child_ptr = M.upload(L.child_ptr);
    if (ell > P.top) {
      const Level& U = P.L(ell - 1);
      const int64_t Bp = (int64_t)U.code.size();
      std::vector<int64_t> z0, z1, y0, y1, x0(Bp, -1), x1(Bp, -1), dxs, dys, dzs(LD.B, -1);
      std::vector<int8_t> zb0, zb1, yb0, yb1, xb0(Bp, 0), xb1(Bp, 0), dxsel, dysel;
      for (int64_t pb = 0; pb < Bp; ++pb) {
        int64_t g1id[2][2] = {{-1, -1}, {-1, -1}}, g2id[2] = {-1, -1};
        for (int64_t c = U.child_ptr[pb]; c < U.child_ptr[pb + 1]; ++c) {
          const int bx = (int)(L.ijk[3 * c] & 1), by = (int)(L.ijk[3 * c + 1] & 1), bz = (int)(L.ijk[3 * c + 2] & 1);
          int64_t& g = g1id[bx][by];
          if (g < 0) {
            g = (int64_t)z0.size();
            z0.push_back(c);
            zb0.push_back((int8_t)bz);
            z1.push_back(-1);
            zb1.push_back(0);
          } else {
            if (z1[g] >= 0) throw EfieError{EFIE_EINVAL, "internal: more than two children share (bx, by)"};
            z1[g] = c;
            zb1[g] = (int8_t)bz;
          }
          dzs[c] = g;
        }
        for (int bx = 0; bx < 2; ++bx)
          for (int by = 0; by < 2; ++by) {
            const int64_t g = g1id[bx][by];
            if (g < 0) continue;
            int64_t& h2 = g2id[bx];
            if (h2 < 0) {
              h2 = (int64_t)y0.size();
              y0.push_back(g);
              yb0.push_back((int8_t)by);
              y1.push_back(-1);
              yb1.push_back(0);
              dxs.push_back(pb);
              dxsel.insert(dxsel.end(), {(int8_t)bx, 0, 0});
            } else {
              y1[h2] = g;
              yb1[h2] = (int8_t)by;
            }
            if ((int64_t)dys.size() <= g) {
              dys.resize(g + 1, -1);
              dysel.resize(3 * (g + 1), 0);
            }
            dys[g] = h2;
            dysel[3 * g + 1] = (int8_t)by;
          }
        for (int bx = 0; bx < 2; ++bx) {
          if (g2id[bx] < 0) continue;
          if (x0[pb] < 0) {
            x0[pb] = g2id[bx];
            xb0[pb] = (int8_t)bx;
          } else {
            x1[pb] = g2id[bx];
            xb1[pb] = (int8_t)bx;
          }
        }
        // a parent without children is a leaf (nonuniform tree): the upward
        // pass writes zeros there, and the leaf's own anterpolation follows
        if (x0[pb] < 0 && !U.leaf[pb]) throw EfieError{EFIE_EINVAL, "internal: parent box without children"};
      }
      LD.ng1 = (int64_t)z0.size();
      LD.ng2 = (int64_t)y0.size();
      LD.uz_s0 = M.upload(z0);
      LD.uz_s1 = M.upload(z1);
      LD.uz_b0 = M.upload(zb0);
      LD.uz_b1 = M.upload(zb1);
      LD.uy_s0 = M.upload(y0);
      LD.uy_s1 = M.upload(y1);
      LD.uy_b0 = M.upload(yb0);
      LD.uy_b1 = M.upload(yb1);
      LD.ux_s0 = M.upload(x0);
      LD.ux_s1 = M.upload(x1);
      LD.ux_b0 = M.upload(xb0);
      LD.ux_b1 = M.upload(xb1);
      LD.dx_src = M.upload(dxs);
      LD.dx_sel = M.upload(dxsel);
      LD.dy_src = M.upload(dys);
      LD.dy_sel = M.upload(dysel);
      LD.dz_src = M.upload(dzs);
    }
    LD.ntiles = (int64_t)L.tile_tgt_ptr.size() - 1;
    // chunks of 16 sources over all tiles (the persistent tensor-core kernel's chunk table)
    // (-1 when a tile has more sources than the table's 16-bit source field takes)
    LD.nq = 0;
    for (int64_t t = 0; t < LD.ntiles && LD.nq >= 0; ++t) {
      const int64_t ns = L.tile_src_ptr[t + 1] - L.tile_src_ptr[t];
      LD.nq = ns > 65536 ? -1 : LD.nq + (ns + 15) / 16;
    }
    if (!L.tct_tgt_ptr.empty()) {
      LD.tct_ntiles = (int64_t)L.tct_tgt_ptr.size() - 1;
      for (int64_t t = 0; t < LD.tct_ntiles; ++t) {
        const int64_t ns = L.tct_src_ptr[t + 1] - L.tct_src_ptr[t];
        LD.tct_max = std::max<int>(LD.tct_max, (int)(L.tct_tgt_ptr[t + 1] - L.tct_tgt_ptr[t]));
        if (LD.tct_nq >= 0) LD.tct_nq = ns > 65536 ? -1 : LD.tct_nq + (ns + 15) / 16;
      }
      {
        std::vector<int16_t> k16;
        std::vector<int64_t> k16_off;
        if (make_index16(L.tct_tgt_ptr, L.tct_src_ptr, L.tct_kidx_off, L.tct_kidx, k16, k16_off)) {
          LD.tct_k16 = M.upload(k16);
          LD.tct_k16_off = M.upload(k16_off);
        }
      }
      LD.tct_tgt_ptr = M.upload(L.tct_tgt_ptr);
      LD.tct_src_ptr = M.upload(L.tct_src_ptr);
      LD.tct_kidx_off = M.upload(L.tct_kidx_off);
      LD.tct_tgt = M.upload(L.tct_tgt);
      LD.tct_src = M.upload(L.tct_src);
      LD.tct_kidx = M.upload(L.tct_kidx);
    }
    for (int64_t t = 0; t < LD.ntiles; ++t)
      LD.max_tile = std::max<int>(LD.max_tile, (int)(L.tile_tgt_ptr[t + 1] - L.tile_tgt_ptr[t]));
    if (LD.ntiles > 0) {
      std::vector<int16_t> k16;
      std::vector<int64_t> k16_off;
      if (make_index16(L.tile_tgt_ptr, L.tile_src_ptr, L.tile_kidx_off, L.tile_kidx, k16, k16_off)) {
        LD.tile_k16 = M.upload(k16);
        LD.tile_k16_off = M.upload(k16_off);
      }
    }
    LD.tile_tgt_ptr = M.upload(L.tile_tgt_ptr);
    LD.tile_src_ptr = M.upload(L.tile_src_ptr);
    LD.tile_kidx_off = M.upload(L.tile_kidx_off);
    LD.tile_tgt = M.upload(L.tile_tgt);
    LD.tile_src = M.upload(L.tile_src);
    LD.tile_kidx = M.upload(L.tile_kidx);
  }
  cuda_check(cudaStreamSynchronize(s), "setup tables");
  phase_done(1);
  // near field (FP64)
  {
    const int64_t BD = P.n_leaves;
    h->d_near_ptr = M.upload(P.near_ptr);
    h->d_near_src = M.upload(P.near_src);
    h->d_blkA_off = M.upload(P.blkA_off);
    h->d_blkV_off = M.upload(P.blkV_off);
    h->d_blkS_off = h->direct ? h->d_blkA_off : h->d_blkV_off;
    std::vector<int32_t> tgt(P.near_src.size());
    for (int64_t x = 0; x < BD; ++x)
      for (int64_t j = P.near_ptr[x]; j < P.near_ptr[x + 1]; ++j) tgt[j] = (int32_t)x;
    NearDev& nd = h->nd;
    nd.V = h->dV;
    nd.T = h->dT;
    nd.area = h->darea;
    nd.k = k;
    nd.n_boxes = BD;
    nd.n_blocks = (int64_t)P.near_src.size();
    nd.near_ptr = h->d_near_ptr;
    nd.near_src = h->d_near_src;
    nd.blk_tgt = M.upload(tgt);
    nd.blkA_off = h->d_blkA_off;
    nd.blkV_off = h->d_blkV_off;
    nd.box_rwg_ptr = h->d_box_rwg_ptr;
    nd.box_tri_ptr = h->d_box_tri_ptr;
    nd.tri_perm = M.upload(P.tri_perm);
    nd.tset_ptr = M.upload(P.tset_ptr);
    nd.tset = M.upload(P.tset);
    nd.rwg_tl = M.upload(P.rwg_tl);
    nd.rwg_loc = M.upload(P.rwg_loc);
    nd.rwg_coef = M.upload(P.rwg_coef);
    {
      // position of each sorted triangle in the A triangle set of its own box
      std::vector<int32_t> tl(P.tri_perm.size(), -1);
      for (int64_t b = 0; b < BD; ++b)
        for (int64_t i = P.box_tri_ptr[b]; i < P.box_tri_ptr[b + 1]; ++i) {
          const auto first = P.tset.begin() + P.tset_ptr[b], last = P.tset.begin() + P.tset_ptr[b + 1];
          const auto it = std::lower_bound(first, last, P.tri_perm[i]);
          if (it != last && *it == P.tri_perm[i]) tl[i] = (int32_t)(it - first);
        }
      nd.tri_tl = M.upload(tl);
    }
    nd.A = M.alloc<double2>(P.nnzA);
    // direct factorization: the scalar part Phi lives on the A blocks
    const int64_t nnzS = h->direct ? P.nnzA : P.nnzV;
    nd.Vn = M.alloc<double2>(nnzS);
    nd.Phi = h->direct ? nd.Vn : nullptr;
    // A: triangle-pair scratch per batch of blocks
    const int64_t nblk = nd.n_blocks;
    const int64_t scr_cap = (int64_t)(1LL << 30) / (10 * 16);  // pairs per batch (~1 GiB)
    double2* scratch = nullptr;
    int64_t* d_scr_off = M.alloc<int64_t>(nblk + 1);
    // T is symmetric: blocks (x, y) with x > y are copied as transposes of
    // (y, x) instead of being integrated.
    std::vector<int64_t> mir_blk, mir_src;
    for (int64_t j = 0; j < nblk; ++j) {
      const int32_t x = tgt[j], y = P.near_src[j];
      if (x <= y) continue;
      int64_t jm = -1;
      for (int64_t q = P.near_ptr[y]; q < P.near_ptr[y + 1]; ++q)
        if (P.near_src[q] == x) jm = q;
      if (jm < 0) throw EfieError{EFIE_EINVAL, "internal: near list is not symmetric"};
      mir_blk.push_back(j);
      mir_src.push_back(jm);
    }
    int64_t max_pairs = 1;
    auto n_pairs = [&](int64_t j) -> int64_t {
      const int32_t x = tgt[j], y = P.near_src[j];
      if (x > y) return 0;
      return (P.tset_ptr[x + 1] - P.tset_ptr[x]) * (P.tset_ptr[y + 1] - P.tset_ptr[y]);
    };
    for (int64_t j = 0; j < nblk; ++j) max_pairs = std::max(max_pairs, n_pairs(j));
    // pairs per batch: ~1 GiB of scratch, less when a device_mem_limit leaves
    // less room (never below the largest block)
    int64_t cap = scr_cap;
    if (M.limit > 0) cap = std::min(cap, (M.limit - M.bytes) / (10 * 16));
    cap = std::max(cap, max_pairs);
    scratch = M.alloc<double2>(10 * cap);
    int64_t j0 = 0;
    std::vector<int64_t> scr_off;
    while (j0 < nblk) {
      scr_off.assign(1, 0);
      int64_t j1 = j0;
      while (j1 < nblk) {
        const int64_t np = n_pairs(j1);
        if (scr_off.back() + np > cap && j1 > j0) break;
        scr_off.push_back(scr_off.back() + np);
        ++j1;
      }
      cuda_check(cudaMemcpy(d_scr_off, scr_off.data(), sizeof(int64_t) * scr_off.size(), cudaMemcpyHostToDevice),
                 "scr_off");
      launch_near_pairs_A(nd, j0, j1 - j0, d_scr_off, scratch, scr_off.back(), s);
      launch_near_combine_A(nd, j0, j1 - j0, d_scr_off, scratch, P.blkA_off[j0],
                            P.blkA_off[j1] - P.blkA_off[j0], s);
      if (!h->direct)
        launch_near_V_pairs(nd, j0, j1 - j0, d_scr_off, scratch, P.blkV_off[j0], P.blkV_off[j1] - P.blkV_off[j0],
                            s);
      cuda_check(cudaStreamSynchronize(s), "near assembly");
      j0 = j1;
    }
    M.release(scratch);
    {
      const int64_t nm = (int64_t)mir_blk.size();
      int64_t* d_mir = M.alloc<int64_t>(2 * std::max<int64_t>(nm, 1));
      if (nm) {
        cuda_check(cudaMemcpy(d_mir, mir_blk.data(), sizeof(int64_t) * nm, cudaMemcpyHostToDevice), "mirror list");
        cuda_check(cudaMemcpy(d_mir + nm, mir_src.data(), sizeof(int64_t) * nm, cudaMemcpyHostToDevice),
                   "mirror list");
      }
      launch_near_mirror(nd.A, nd.blkA_off, nd.box_rwg_ptr, nd.blk_tgt, nd.near_src, d_mir, d_mir + nm, nm, s);
      if (h->direct)
        launch_near_mirror(nd.Vn, nd.blkA_off, nd.box_rwg_ptr, nd.blk_tgt, nd.near_src, d_mir, d_mir + nm, nm, s);
      else
        launch_near_mirror(nd.Vn, nd.blkV_off, nd.box_tri_ptr, nd.blk_tgt, nd.near_src, d_mir, d_mir + nm, nm, s);
      cuda_check(cudaStreamSynchronize(s), "near mirror");
      M.release(d_mir);
    }
    if (h->precision == EFIE_MIXED) {
      // keep the FP64-assembled values as double-float pairs (in place)
      launch_split_df(nd.A, P.nnzA, s);
      launch_split_df(nd.Vn, nnzS, s);
      cuda_check(cudaStreamSynchronize(s), "near split");
      h->near_df = true;
    }
  }
  cuda_check(cudaStreamSynchronize(s), "near setup");
  phase_done(2);
  // far products
  if (h->opt.precond == EFIE_PRECOND_LEARNED && h->opt.weights_path) {
    std::vector<float> w;
    if (read_weights(h->opt.weights_path, w)) net_activate(h, w, false);  // else: plain GMRES (fallback flag)
  }
  build_far<double>(h, h->f64, s);
  std::vector<double2*> K64 = build_kernel_spectra64(h, s);
  build_spectra<double>(h, h->f64, K64, s);
  if (h->precision == EFIE_MIXED) {
    build_far<float>(h, h->f32, s);
    build_spectra<float>(h, h->f32, K64, s);
  }
  if (h->dyadic)
    for (int c = 0; c < 6; ++c) {
      std::vector<double2*> KH = build_kernel_spectra64(h, s, c);
      build_spectra<double>(h, h->f64, KH, s, c);
      if (h->precision == EFIE_MIXED) build_spectra<float>(h, h->f32, KH, s, c);
    }
  cuda_check(cudaStreamSynchronize(s), "setup");
  phase_done(3);
}

// ------------------------------------------------------------- GMRES
// Device buffers of one call, released on every exit (also when an
// allocation or a launch throws).
struct Workspace {
  DevMem& M;
  std::vector<void*> p;
  template <typename T>
  T* take(int64_t n) {
    T* q = M.alloc<T>(n);
    p.push_back(q);
    return q;
  }
  ~Workspace() {
    for (void* q : p) M.release(q);
  }
};

struct Givens {
  std::vector<std::complex<double>> H, cs, sn, g;
};

int solve_impl(efie_handle* h, const double2* b, double2* x, int n_rhs, double tol, efie_solve_info* info,
               cudaStream_t s, double2* rec = nullptr, int rec_cycles = 0) {
  if (!(tol > 0)) throw EfieError{EFIE_EINVAL, "tol must be positive"};
  // the working-precision (estimated and restart) residuals aim at tol/2 so that
  // the final FP64 true residual meets tol
  const double tol_in = 0.5 * tol;
  const int64_t N = h->plan.g.N;
  const int m = h->opt.gmres_restart;
  const int max_it = rec ? m * rec_cycles : h->opt.max_iters;
  int cycle = 0;
  Workspace ws{h->mem, {}};
  double2* Vb = ws.take<double2>((int64_t)n_rhs * (m + 1) * N);
  const bool use_pc = h->net != nullptr && h->opt.precond == EFIE_PRECOND_LEARNED;
  double2* Zb = use_pc ? ws.take<double2>((int64_t)n_rhs * m * N) : nullptr;
  std::vector<int> pc_fallback(n_rhs, 0);
  double2* wv = ws.take<double2>((int64_t)n_rhs * N);
  double2* rv = ws.take<double2>((int64_t)n_rhs * N);
  double2* dh = ws.take<double2>((int64_t)n_rhs * (m + 1));
  double2* dh2 = ws.take<double2>((int64_t)n_rhs * (m + 1));
  double* dn = ws.take<double>(n_rhs);
  int* dact = ws.take<int>(n_rhs);
  const int64_t ldr = (int64_t)(m + 1) * N;
  std::vector<double> bnorm(n_rhs), nrm(n_rhs);
  std::vector<int> its(n_rhs, 0), conv(n_rhs, 0), act(n_rhs, 1);
  std::vector<std::complex<double>> hh((size_t)n_rhs * (m + 1)), hh2((size_t)n_rhs * (m + 1));
  auto d2h = [&](std::vector<std::complex<double>>& dst, const double2* src, int64_t n) {
    cuda_check(cudaMemcpyAsync(dst.data(), src, sizeof(double2) * n, cudaMemcpyDeviceToHost, s), "d2h");
    cuda_check(cudaStreamSynchronize(s), "sync");
  };
  auto norms = [&](const double2* v, int64_t ld, std::vector<double>& out) {
    launch_norms(v, ld, N, n_rhs, dn, s);
    cuda_check(cudaMemcpyAsync(out.data(), dn, sizeof(double) * n_rhs, cudaMemcpyDeviceToHost, s), "d2h");
    cuda_check(cudaStreamSynchronize(s), "sync");
    for (auto& v2 : out) v2 = std::sqrt(v2);
  };
  cuda_check(cudaMemsetAsync(x, 0, sizeof(double2) * n_rhs * N, s), "x0");
  cuda_check(cudaMemsetAsync(Vb, 0, sizeof(double2) * n_rhs * ldr, s), "basis");
  norms(b, N, bnorm);
  cuda_check(cudaMemcpyAsync(rv, b, sizeof(double2) * n_rhs * N, cudaMemcpyDeviceToDevice, s), "r0");
  std::vector<double> beta(n_rhs);
  for (int r = 0; r < n_rhs; ++r) {
    beta[r] = bnorm[r];
    if (bnorm[r] == 0) {
      act[r] = 0;
      conv[r] = 1;
    }
  }
  std::vector<std::vector<std::complex<double>>> H(n_rhs), cs(n_rhs), sn(n_rhs), gg(n_rhs);
  std::vector<int> floor_hits(n_rhs, 0), refine(n_rhs, 0);
  while (true) {
    bool any = false;
    for (int r = 0; r < n_rhs; ++r) {
      if (act[r] && (beta[r] / bnorm[r] <= tol_in || its[r] >= max_it)) act[r] = 0;
      any |= act[r] != 0;
    }
    if (!any) break;
    cuda_check(cudaMemcpyAsync(dact, act.data(), sizeof(int) * n_rhs, cudaMemcpyHostToDevice, s), "act");
    // V0 = r / beta
    for (int r = 0; r < n_rhs; ++r) {
      H[r].assign((size_t)(m + 1) * m, 0.0);
      cs[r].assign(m, 0.0);
      sn[r].assign(m, 0.0);
      gg[r].assign(m + 1, 0.0);
      gg[r][0] = beta[r];
      hh[r] = act[r] ? 1.0 / beta[r] : 0.0;
    }
    for (int r = 0; r < n_rhs; ++r) cuda_check(cudaMemsetAsync(Vb + r * ldr, 0, sizeof(double2) * N, s), "v0");
    cuda_check(cudaMemcpyAsync(dh, hh.data(), sizeof(double2) * n_rhs, cudaMemcpyHostToDevice, s), "h");
    launch_multiaxpy(rv, N, 0, 1, dh, 1, Vb, ldr, N, n_rhs, dact, 1.0, s);
    std::vector<int> kdim(n_rhs, 0), inner(n_rhs, 0), est_conv(n_rhs, 0);
    for (int r = 0; r < n_rhs; ++r) inner[r] = act[r];
    for (int k = 0; k < m; ++k) {
      bool anyin = false;
      for (int r = 0; r < n_rhs; ++r) anyin |= inner[r] != 0;
      if (!anyin) break;
      std::vector<int> ia(inner);
      cuda_check(cudaMemcpyAsync(dact, ia.data(), sizeof(int) * n_rhs, cudaMemcpyHostToDevice, s), "act");
      // z_k = M(v_k) (flexible right preconditioner), w = T z_k
      const double2* zk = Vb + (int64_t)k * N;
      int64_t ldz = ldr;
      if (use_pc) {
        KScope ks(h, K_PRECOND, s, 6);
        for (int r = 0; r < n_rhs; ++r) {
          double2* zr = Zb + (int64_t)r * m * N + (int64_t)k * N;
          const double2* vr = Vb + r * ldr + (int64_t)k * N;
          if (inner[r] && !pc_fallback[r]) {
            efie::nn_forward(*h->net, vr, zr, false, s);
            // non-finite network output: identity for the rest of this solve
            double nz = 0;
            launch_norms(zr, N, N, 1, dn, s);
            cuda_check(cudaMemcpyAsync(&nz, dn, sizeof(double), cudaMemcpyDeviceToHost, s), "d2h");
            cuda_check(cudaStreamSynchronize(s), "sync");
            if (!std::isfinite(nz) || nz == 0) pc_fallback[r] = 1;
          }
          if (!inner[r] || pc_fallback[r])
            cuda_check(cudaMemcpyAsync(zr, vr, sizeof(double2) * N, cudaMemcpyDeviceToDevice, s), "copy");
        }
        zk = Zb + (int64_t)k * N;
        ldz = (int64_t)m * N;
      }
      do_matvec(h, zk, ldz, wv, nullptr, nullptr, N, n_rhs, false, s);
      // CGS2
      KScope ks(h, K_KRYLOV, s, 5);
      launch_multidot(Vb, ldr, N, k + 1, wv, N, N, n_rhs, dact, dh, s);
      launch_multiaxpy(Vb, ldr, N, k + 1, dh, k + 1, wv, N, N, n_rhs, dact, -1.0, s);
      launch_multidot(Vb, ldr, N, k + 1, wv, N, N, n_rhs, dact, dh2, s);
      launch_multiaxpy(Vb, ldr, N, k + 1, dh2, k + 1, wv, N, N, n_rhs, dact, -1.0, s);
      d2h(hh, dh, (int64_t)n_rhs * (k + 1));
      d2h(hh2, dh2, (int64_t)n_rhs * (k + 1));
      norms(wv, N, nrm);
      std::vector<std::complex<double>> sc((size_t)n_rhs, 0.0);
      for (int r = 0; r < n_rhs; ++r) {
        if (!inner[r]) continue;
        for (int i = 0; i <= k; ++i) H[r][(size_t)i * m + k] = hh[(size_t)r * (k + 1) + i] + hh2[(size_t)r * (k + 1) + i];
        H[r][(size_t)(k + 1) * m + k] = nrm[r];
        sc[r] = nrm[r] > 0 ? 1.0 / nrm[r] : 0.0;
        // Givens: G = [[conj(c), conj(s)], [-s, c]], c = a/den, s = b/den
        for (int i = 0; i < k; ++i) {
          auto t = std::conj(cs[r][i]) * H[r][(size_t)i * m + k] + std::conj(sn[r][i]) * H[r][(size_t)(i + 1) * m + k];
          H[r][(size_t)(i + 1) * m + k] = -sn[r][i] * H[r][(size_t)i * m + k] + cs[r][i] * H[r][(size_t)(i + 1) * m + k];
          H[r][(size_t)i * m + k] = t;
        }
        auto a = H[r][(size_t)k * m + k], bb = H[r][(size_t)(k + 1) * m + k];
        double den = std::sqrt(std::norm(a) + std::norm(bb));
        cs[r][k] = den > 0 ? a / den : 1.0;
        sn[r][k] = den > 0 ? bb / den : 0.0;
        H[r][(size_t)k * m + k] = den;
        H[r][(size_t)(k + 1) * m + k] = 0.0;
        gg[r][k + 1] = -sn[r][k] * gg[r][k];
        gg[r][k] = std::conj(cs[r][k]) * gg[r][k];
        its[r]++;
        kdim[r] = k + 1;
        if (std::abs(gg[r][k + 1]) / bnorm[r] <= tol_in) est_conv[r] = 1;
        if (est_conv[r] || its[r] >= max_it || nrm[r] == 0) inner[r] = 0;
      }
      // v_{k+1} = w / ||w||
      std::vector<std::complex<double>> scv(sc);
      cuda_check(cudaMemcpyAsync(dh, scv.data(), sizeof(double2) * n_rhs, cudaMemcpyHostToDevice, s), "h");
      if (k + 1 <= m) {
        for (int r = 0; r < n_rhs; ++r)
          cuda_check(cudaMemsetAsync(Vb + r * ldr + (int64_t)(k + 1) * N, 0, sizeof(double2) * N, s), "vk");
        launch_multiaxpy(wv, N, 0, 1, dh, 1, Vb + (int64_t)(k + 1) * N, ldr, N, n_rhs, dact, 1.0, s);
      }
    }
    // x += V y (y from the triangular system)
    std::vector<std::complex<double>> yv((size_t)n_rhs * m, 0.0);
    for (int r = 0; r < n_rhs; ++r) {
      int kd = kdim[r];
      for (int i = kd - 1; i >= 0; --i) {
        auto sacc = gg[r][i];
        for (int j = i + 1; j < kd; ++j) sacc -= H[r][(size_t)i * m + j] * yv[(size_t)r * m + j];
        yv[(size_t)r * m + i] = sacc / H[r][(size_t)i * m + i];
      }
    }
    cuda_check(cudaMemcpyAsync(dh, yv.data(), sizeof(double2) * n_rhs * m, cudaMemcpyHostToDevice, s), "y");
    cuda_check(cudaMemcpyAsync(dact, act.data(), sizeof(int) * n_rhs, cudaMemcpyHostToDevice, s), "act");
    if (use_pc)
      launch_multiaxpy(Zb, (int64_t)m * N, N, m, dh, m, x, N, N, n_rhs, dact, 1.0, s);
    else
      launch_multiaxpy(Vb, ldr, N, m, dh, m, x, N, N, n_rhs, dact, 1.0, s);
    if (rec && cycle < rec_cycles)
      cuda_check(cudaMemcpyAsync(rec + (int64_t)cycle * n_rhs * N, x, sizeof(double2) * n_rhs * N,
                                 cudaMemcpyDeviceToDevice, s), "record");
    ++cycle;
    // restart residual r = b - T x: working precision, or the FP64 product
    // once a right-hand side of a mixed handle has reached the working
    // precision's accuracy floor (mixed-precision iterative refinement: the
    // next cycles solve T_mixed d = b - T_fp64 x, whose fixed point is the
    // FP64 solution)
    bool use64 = false;
    for (int r = 0; r < n_rhs; ++r) use64 |= act[r] && refine[r];
    do_matvec(h, x, N, wv, nullptr, nullptr, N, n_rhs, use64, s);
    launch_lincomb(b, wv, 1.0, -1.0, rv, (int64_t)n_rhs * N, s);
    std::vector<double> beta_prev(beta);
    norms(rv, N, beta);
    // a flexible cycle that made no progress (< 1%) hands this right-hand side
    // back to plain GMRES
    if (use_pc)
      for (int r = 0; r < n_rhs; ++r)
        if (act[r] && !pc_fallback[r] && beta[r] > 0.99 * beta_prev[r]) pc_fallback[r] = 1;
    // accuracy floor: the cycle met the tolerance in its own arithmetic but
    // the recomputed residual did not.  A mixed handle then switches that
    // right-hand side to FP64 restart residuals (refinement, from this
    // restart on); otherwise, twice in a row, further cycles cannot lower it,
    // so stop and let the FP64 true residual below decide convergence
    bool newly = false;
    for (int r = 0; r < n_rhs; ++r) {
      if (!act[r]) continue;
      if (est_conv[r] && beta[r] / bnorm[r] > tol_in) {
        if (h->precision == EFIE_MIXED && !refine[r]) {
          refine[r] = 1;
          newly = !use64 || newly;
        } else if (++floor_hits[r] >= 2) {
          act[r] = 0;
        }
      } else {
        floor_hits[r] = 0;
      }
    }
    if (newly) {
      do_matvec(h, x, N, wv, nullptr, nullptr, N, n_rhs, true, s);
      launch_lincomb(b, wv, 1.0, -1.0, rv, (int64_t)n_rhs * N, s);
      norms(rv, N, beta);
    }
  }
  // true residual with the FP64 fast matvec
  do_matvec(h, x, N, wv, nullptr, nullptr, N, n_rhs, true, s);
  launch_lincomb(b, wv, 1.0, -1.0, rv, (int64_t)n_rhs * N, s);
  norms(rv, N, nrm);
  int ret = EFIE_OK;
  for (int r = 0; r < n_rhs; ++r) {
    double rel = bnorm[r] > 0 ? nrm[r] / bnorm[r] : 0.0;
    conv[r] = rel <= tol;
    if (!conv[r]) ret = EFIE_NOT_CONVERGED;
    if (info) {
      info[r].iterations = its[r];
      info[r].true_rel_residual = rel;
      info[r].converged = conv[r];
      info[r].precond_fallback = (h->opt.precond == EFIE_PRECOND_LEARNED && (!use_pc || pc_fallback[r])) ? 1 : 0;
    }
  }
  return ret;
}

template <typename F>
int guarded(efie_handle* h, F&& f) {
  try {
    return f();
  } catch (const EfieError& e) {
    set_err(h, e);
    return e.code;
  } catch (const std::bad_alloc&) {
    set_err(h, EfieError{EFIE_ENOMEM, "host allocation failed"});
    return EFIE_ENOMEM;
  } catch (const std::exception& e) {
    set_err(h, EfieError{EFIE_EINVAL, e.what()});
    return EFIE_EINVAL;
  }
}

void fill_plan_info(const Plan& P, efie_plan_info_t* info, efie_level_info_t* lv, int max_levels) {
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->n_unknowns = P.g.N;
    info->n_triangles = P.g.nt;
    info->depth = P.D;
    info->top_level = P.top;
    info->n_levels = P.n_levels;
    info->p = P.p;
    for (int d = 0; d < 3; ++d) info->root_lo[d] = P.root_lo[d];
    info->root_edge = P.root_edge;
    info->near_nnz_A = P.nnzA;
    info->near_nnz_V = P.nnzV;
    int64_t bytes = (P.nnzA + P.nnzV) * 16;
    for (const Level& L : P.lv) {
      int64_t n3 = (int64_t)L.nfft * L.nfft * L.nfft;
      bytes += n3 * (int64_t)(L.offsets.size() / 3) * 16;
    }
    info->device_bytes = bytes;
    info->moment_entries_rwg = P.mom_rwg.off.empty() ? 0 : P.mom_rwg.off.back() / 3;
    info->moment_entries_tri = P.mom_tri.off.empty() ? 0 : P.mom_tri.off.back();
  }
  if (lv) {
    int i = 0;
    for (int ell = P.D; ell >= P.top && i < max_levels; --ell, ++i) {
      const Level& L = P.L(ell);
      efie_level_info_t& o = lv[i];
      o.level = ell;
      o.s = L.s;
      o.sb = L.sb;
      o.sp = L.sp;
      o.shat = L.shat;
      o.nfft = L.nfft;
      o.n_boxes = (int64_t)L.code.size();
      o.n_far_pairs = (int64_t)L.il_src.size();
      o.n_offsets = (int64_t)L.offsets.size() / 3;
      o.h = L.h;
      o.delta = L.delta;
      o.Delta = L.Delta;
    }
  }
}

}  // namespace

namespace {
// RWG adjacency: neighbours share a triangle c, sign sigma_{m,c} sigma_{n,c}
void build_nn_graph(efie_handle* h) {
  if (!h->g_nbr.empty()) return;
  const Geometry& g = h->plan.g;
  const int64_t N = g.N, nt = g.nt;
  std::vector<int32_t> tr(3 * nt, -1);
  std::vector<float> ts(3 * nt, 0.f);
  std::vector<int> cnt(nt, 0);
  for (int64_t m = 0; m < N; ++m)
    for (int sd = 0; sd < 2; ++sd) {
      int32_t t = g.tri_pm[2 * m + sd];
      tr[3 * t + cnt[t]] = (int32_t)m;
      ts[3 * t + cnt[t]] = sd == 0 ? 1.f : -1.f;
      cnt[t]++;
    }
  h->g_nbr.assign(4 * N, -1);
  h->g_sgn.assign(4 * N, 0.f);
  std::vector<int> nc(N, 0);
  for (int64_t t = 0; t < nt; ++t)
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        if (a == b || tr[3 * t + a] < 0 || tr[3 * t + b] < 0) continue;
        int32_t m = tr[3 * t + a];
        if (nc[m] >= 4) continue;
        h->g_nbr[4 * m + nc[m]] = tr[3 * t + b];
        h->g_sgn[4 * m + nc[m]] = ts[3 * t + a] * ts[3 * t + b];
        nc[m]++;
      }
  h->g_len.resize(N);
  double mean = 0;
  for (int64_t m = 0; m < N; ++m) {
    double d2 = 0;
    for (int d = 0; d < 3; ++d) {
      double t = g.V[3 * g.edge[2 * m] + d] - g.V[3 * g.edge[2 * m + 1] + d];
      d2 += t * t;
    }
    h->g_len[m] = (float)std::sqrt(d2);
    mean += h->g_len[m];
  }
  mean /= (double)N;
  for (auto& l : h->g_len) l = (float)(l / mean);
}

void net_activate(efie_handle* h, const std::vector<float>& params, bool training) {
  build_nn_graph(h);
  if (h->net) {
    efie::nn_delete(h->net);
    h->net = nullptr;
  }
  h->net = efie::nn_new();
  efie::nn_setup(*h->net, h->plan.g.N, h->g_nbr, h->g_sgn, h->g_len, params, training);
  h->net_params = params;
  h->net_training = training;
}

bool read_weights(const char* path, std::vector<float>& p) {
  FILE* f = std::fopen(path, "rb");
  if (!f) return false;
  char magic[8] = {0};
  int32_t n = 0;
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "EFIENN01", 8) == 0 &&
            std::fread(&n, sizeof(n), 1, f) == 1 && n == efie::nn_param_count();
  if (ok) {
    p.resize(n);
    ok = std::fread(p.data(), sizeof(float), n, f) == (size_t)n;
  }
  std::fclose(f);
  for (float v : p)
    if (!std::isfinite(v)) ok = false;
  return ok;
}
}  // namespace

namespace efie {
int handle_rhs_args(const efie_handle* h, const double** V, const int32_t** T, const double** area,
                    const int32_t** tri_pm, const int32_t** free_pm, int64_t* N, double* k, int* device) {
  if (!h) return EFIE_EINVAL;
  *device = h->device;
  *V = h->dV;
  *T = h->dT;
  *area = h->darea;
  *tri_pm = h->dtri_pm;
  *free_pm = h->dfree_pm;
  *N = h->plan.g.N;
  *k = h->plan.k;
  return EFIE_OK;
}
void handle_set_error(efie_handle* h, const char* msg) {
  if (h) h->err = msg;
  g_last_error = msg;
}
}  // namespace efie

// ================================================================= C ABI
namespace {
AdaptiveOptions adaptive_options(const efie_tree_options* topt) {
  AdaptiveOptions o;
  if (topt) {
    o.max_elems = topt->max_elems;
    o.max_prot = topt->max_prot;
    o.top = topt->top;
    o.n_splines = topt->n_splines;
    o.max_depth = topt->max_depth > 0 ? topt->max_depth : 30;
    if (!(o.max_prot >= 0)) throw EfieError{EFIE_EINVAL, "max_prot must be >= 0"};
  }
  return o;
}

}  // namespace

extern "C" {

int efie_plan(const efie_mesh* mesh, double wavenumber, int spline_degree, double grid_spacing, int levels,
              const efie_options* opt, efie_plan_info_t* info, efie_level_info_t* levels_out, int max_levels) {
  return guarded(nullptr, [&] {
    check_mesh(mesh);
    efie_options o = defaults(opt);
    Plan P;
    build_plan(P, mesh->xyz, mesh->n_vertices, mesh->tri, mesh->n_triangles, wavenumber, spline_degree,
               grid_spacing, levels, o.n_splines, false);
    fill_plan_info(P, info, levels_out, max_levels);
    return EFIE_OK;
  });
}

int efie_plan_adaptive(const efie_mesh* mesh, double wavenumber, int spline_degree, const efie_tree_options* topt,
                       efie_adaptive_level_t* levels_out, int max_levels, int32_t* n_levels, int64_t* near_pairs_rwg,
                       int64_t* near_pairs_tri) {
  return guarded(nullptr, [&] {
    check_mesh(mesh);
    if (max_levels < 0) throw EfieError{EFIE_EINVAL, "max_levels < 0"};
    // the plan the device pipeline runs (efie_setup_adaptive): its
    // interaction lists, leaves and near blocks are what is reported
    Plan P;
    build_plan_adaptive(P, mesh->xyz, mesh->n_vertices, mesh->tri, mesh->n_triangles, wavenumber, spline_degree,
                        adaptive_options(topt), false);
    const int nl = (int)P.lv.size();
    if (n_levels) *n_levels = nl;
    if (near_pairs_rwg) *near_pairs_rwg = P.nnzA;
    if (near_pairs_tri) *near_pairs_tri = P.nnzV;
    if (levels_out)
      for (int i = 0; i < std::min(nl, max_levels); ++i) {
        const Level& L = P.lv[i];
        efie_adaptive_level_t& out = levels_out[i];
        out.level = L.level;
        out.s = L.s;
        out.sb = L.sb;
        out.sp = L.sp;
        out.shat = L.shat;
        out.n_boxes = (int64_t)L.code.size();
        const int64_t l0 = P.level_leaf_ptr[i], l1 = P.level_leaf_ptr[i + 1];
        out.n_leaves = l1 - l0;
        out.n_far_pairs = (int64_t)L.il_src.size();
        out.n_leaf_rwg = P.box_rwg_ptr[l1] - P.box_rwg_ptr[l0];
        out.n_leaf_tri = P.box_tri_ptr[l1] - P.box_tri_ptr[l0];
        out.h = L.h;
        out.delta = L.delta;
      }
    return EFIE_OK;
  });
}

int efie_plan_adaptive_near(const efie_mesh* mesh, double wavenumber, int spline_degree,
                            const efie_tree_options* topt, int64_t* n_leaves, int64_t* nnz, int32_t* leaf_level,
                            int64_t* leaf_ijk, int64_t leaf_cap, int64_t* near_ptr, int32_t* near_src,
                            int64_t near_cap) {
  return guarded(nullptr, [&] {
    check_mesh(mesh);
    AdaptivePlan A;
    build_adaptive_plan(A, mesh->xyz, mesh->n_vertices, mesh->tri, mesh->n_triangles, wavenumber, spline_degree,
                        adaptive_options(topt));
    const int64_t NL = (int64_t)A.leaf_level.size(), nz = (int64_t)A.near_src.size();
    if (n_leaves) *n_leaves = NL;
    if (nnz) *nnz = nz;
    if ((leaf_level || leaf_ijk) && leaf_cap < NL) throw EfieError{EFIE_EINVAL, "leaf_cap too small"};
    if (near_ptr && leaf_cap < NL + 1)
      throw EfieError{EFIE_EINVAL, "leaf_cap too small for near_ptr (needs n_leaves + 1)"};
    if (near_src && near_cap < nz) throw EfieError{EFIE_EINVAL, "near_cap too small"};
    for (int64_t x = 0; x < NL; ++x) {
      if (leaf_level) leaf_level[x] = A.leaf_level[x];
      if (leaf_ijk)
        for (int d = 0; d < 3; ++d) leaf_ijk[3 * x + d] = A.lv[A.leaf_level[x] - A.top].key[A.leaf_box[x]][d];
    }
    if (near_ptr) std::memcpy(near_ptr, A.near_ptr.data(), sizeof(int64_t) * (NL + 1));
    if (near_src) std::memcpy(near_src, A.near_src.data(), sizeof(int32_t) * nz);
    return EFIE_OK;
  });
}

int efie_plan_adaptive_moments(const efie_mesh* mesh, double wavenumber, int spline_degree,
                               const efie_tree_options* topt, int kind, const int32_t* ids, int64_t n_ids,
                               double* out, int64_t out_len, int64_t* out_needed, int32_t* level_out,
                               int32_t* sp_out) {
  return guarded(nullptr, [&] {
    check_mesh(mesh);
    if (kind != 0 && kind != 1) throw EfieError{EFIE_EINVAL, "kind must be 0 (RWG) or 1 (triangle)"};
    if (n_ids < 0 || (n_ids > 0 && !ids)) throw EfieError{EFIE_EINVAL, "ids is NULL"};
    // the moments the device pipeline uploads (efie_setup_adaptive)
    Plan A;
    build_plan_adaptive(A, mesh->xyz, mesh->n_vertices, mesh->tri, mesh->n_triangles, wavenumber, spline_degree,
                        adaptive_options(topt), true);
    const int ncomp = kind == 0 ? 3 : 1;
    const std::vector<int32_t>& perm = kind == 0 ? A.rwg_perm : A.tri_perm;
    const std::vector<int32_t>& leaf = kind == 0 ? A.rwg_box : A.tri_box;
    const MomentBlocks& MB = kind == 0 ? A.mom_rwg : A.mom_tri;
    std::vector<int64_t> rank(perm.size(), -1);
    for (size_t i = 0; i < perm.size(); ++i) rank[perm[i]] = (int64_t)i;
    int64_t need = 0;
    for (int64_t j = 0; j < n_ids; ++j) {
      if (ids[j] < 0 || ids[j] >= (int64_t)rank.size()) throw EfieError{EFIE_EINVAL, "index out of range"};
      const Level& L = A.L(A.leaf_level[leaf[rank[ids[j]]]]);
      need += (int64_t)ncomp * L.sp * L.sp * L.sp;
    }
    if (out_needed) *out_needed = need;
    if (out && out_len < need) throw EfieError{EFIE_EINVAL, "output buffer too small"};
    int64_t pos = 0;
    for (int64_t j = 0; j < n_ids; ++j) {
      const int64_t i = rank[ids[j]];
      const int lvl = A.leaf_level[leaf[i]];
      const int sp = A.L(lvl).sp;
      if (level_out) level_out[j] = lvl;
      if (sp_out) sp_out[j] = sp;
      if (out) {
        double* dst = out + pos;
        std::fill(dst, dst + (int64_t)ncomp * sp * sp * sp, 0.0);
        const int* b = &MB.base[3 * i];
        const int* e = &MB.ext[3 * i];
        const double* src = &MB.data[MB.off[i]];
        for (int c = 0; c < ncomp; ++c)
          for (int a0 = 0; a0 < e[0]; ++a0)
            for (int a1 = 0; a1 < e[1]; ++a1)
              for (int a2 = 0; a2 < e[2]; ++a2)
                dst[(((int64_t)c * sp + b[0] + a0) * sp + b[1] + a1) * sp + b[2] + a2] =
                    src[(((int64_t)c * e[0] + a0) * e[1] + a1) * e[2] + a2];
      }
      pos += (int64_t)ncomp * sp * sp * sp;
    }
    return EFIE_OK;
  });
}

int efie_plan_matrix(const efie_mesh* mesh, double wavenumber, int spline_degree, double grid_spacing,
                     int levels, const efie_options* opt, int level, int which, double* out, int64_t out_len,
                     int32_t* rows, int32_t* cols) {
  return guarded(nullptr, [&] {
    check_mesh(mesh);
    efie_options o = defaults(opt);
    Plan P;
    build_plan(P, mesh->xyz, mesh->n_vertices, mesh->tri, mesh->n_triangles, wavenumber, spline_degree,
               grid_spacing, levels, o.n_splines, false);
    if (level < P.top || level > P.D) throw EfieError{EFIE_EINVAL, "level is not a grid level"};
    const Level& L = P.L(level);
    const std::vector<double>* M = nullptr;
    int r = 0, c = 0;
    if (which == 0) {
      M = &L.P;
      r = L.shat;
      c = L.sp;
    } else if (which == 1 || which == 2) {
      if (level == P.top) throw EfieError{EFIE_EINVAL, "no transfer above the top grid level"};
      M = which == 1 ? &L.CL : &L.CR;
      r = P.L(level - 1).sp;
      c = L.sp;
    } else {
      throw EfieError{EFIE_EINVAL, "which must be 0, 1 or 2"};
    }
    if (rows) *rows = r;
    if (cols) *cols = c;
    if (out) {
      if (out_len < (int64_t)M->size()) throw EfieError{EFIE_EINVAL, "output buffer too small"};
      std::memcpy(out, M->data(), sizeof(double) * M->size());
    }
    return EFIE_OK;
  });
}

int efie_plan_moments(const efie_mesh* mesh, double wavenumber, int spline_degree, double grid_spacing,
                      int levels, const efie_options* opt, int kind, const int32_t* ids, int64_t n_ids,
                      double* out, int64_t out_len, int32_t* sp_out) {
  return guarded(nullptr, [&] {
    check_mesh(mesh);
    if (kind < 0 || kind > 2) throw EfieError{EFIE_EINVAL, "kind must be 0 (RWG), 1 (triangle) or 2 (divergence)"};
    if (n_ids < 0 || (n_ids > 0 && !ids)) throw EfieError{EFIE_EINVAL, "ids is NULL"};
    efie_options o = defaults(opt);
    Plan P;
    build_plan(P, mesh->xyz, mesh->n_vertices, mesh->tri, mesh->n_triangles, wavenumber, spline_degree,
               grid_spacing, levels, o.n_splines, true, kind == 2);
    const int sp = P.L(P.D).sp;
    const int ncomp = kind == 0 ? 3 : 1;
    if (sp_out) *sp_out = sp;
    if (!out) return EFIE_OK;
    const int64_t per = (int64_t)ncomp * sp * sp * sp;
    if (out_len < n_ids * per) throw EfieError{EFIE_EINVAL, "output buffer too small"};
    const std::vector<int32_t>& perm = kind == 1 ? P.tri_perm : P.rwg_perm;
    const MomentBlocks& MB = kind == 0 ? P.mom_rwg : kind == 1 ? P.mom_tri : P.mom_div;
    std::vector<int64_t> rank(perm.size(), -1);
    for (size_t i = 0; i < perm.size(); ++i) rank[perm[i]] = (int64_t)i;
    std::fill(out, out + n_ids * per, 0.0);
    for (int64_t j = 0; j < n_ids; ++j) {
      if (ids[j] < 0 || ids[j] >= (int64_t)rank.size()) throw EfieError{EFIE_EINVAL, "index out of range"};
      const int64_t i = rank[ids[j]];
      const int* b = &MB.base[3 * i];
      const int* e = &MB.ext[3 * i];
      const double* src = &MB.data[MB.off[i]];
      double* dst = out + j * per;
      for (int c = 0; c < ncomp; ++c)
        for (int a0 = 0; a0 < e[0]; ++a0)
          for (int a1 = 0; a1 < e[1]; ++a1)
            for (int a2 = 0; a2 < e[2]; ++a2)
              dst[(((int64_t)c * sp + b[0] + a0) * sp + b[1] + a1) * sp + b[2] + a2] =
                  src[(((int64_t)c * e[0] + a0) * e[1] + a1) * e[2] + a2];
    }
    return EFIE_OK;
  });
}

namespace {
int setup_handle(const efie_options* opt, efie_handle** out, const std::function<void(efie_handle*)>& run) {
  if (!out) {
    g_last_error = "out is NULL";
    return EFIE_EINVAL;
  }
  *out = nullptr;
  efie_handle* h = new (std::nothrow) efie_handle();
  if (!h) {
    g_last_error = "host allocation failed";
    return EFIE_ENOMEM;
  }
  h->opt = defaults(opt);
  h->precision = h->opt.precision;
  int rc = guarded(h, [&] {
    run(h);
    return EFIE_OK;
  });
  if (rc != EFIE_OK) {
    g_last_error = h->err;
    delete h;
    return rc;
  }
  *out = h;
  return EFIE_OK;
}
}  // namespace

int efie_setup(const efie_mesh* mesh, double wavenumber, int spline_degree, double grid_spacing, int levels,
               const efie_options* opt, efie_handle** out) {
  return setup_handle(opt, out, [&](efie_handle* h) {
    setup_impl(h, mesh, wavenumber, spline_degree, grid_spacing, levels);
  });
}

int efie_setup_adaptive(const efie_mesh* mesh, double wavenumber, int spline_degree, const efie_tree_options* topt,
                        const efie_options* opt, efie_handle** out) {
  return setup_handle(opt, out, [&](efie_handle* h) {
    const AdaptiveOptions o = adaptive_options(topt);
    setup_impl(h, mesh, wavenumber, spline_degree, 0.0, 0, &o);
  });
}

int efie_num_unknowns(const efie_handle* h, int64_t* n) {
  if (!h || !n) return EFIE_EINVAL;
  *n = h->plan.g.N;
  return EFIE_OK;
}

int efie_plan_info(const efie_handle* h, efie_plan_info_t* info) {
  if (!h || !info) return EFIE_EINVAL;
  fill_plan_info(h->plan, info, nullptr, 0);
  info->device_bytes = h->mem.bytes;
  if (h->direct) {
    // the scalar part is Phi on the RWG pairs of the A blocks, its moments per RWG
    info->near_nnz_V = info->near_nnz_A;
    const MomentBlocks& MD = h->plan.mom_div;
    info->moment_entries_tri = MD.off.empty() ? 0 : MD.off.back();
  }
  return EFIE_OK;
}

int efie_rwg_edges(const efie_handle* h, int32_t* edge_vertices, int32_t* tri_pm) {
  if (!h) return EFIE_EINVAL;
  const Geometry& g = h->plan.g;
  if (edge_vertices) std::memcpy(edge_vertices, g.edge.data(), sizeof(int32_t) * g.edge.size());
  if (tri_pm) std::memcpy(tri_pm, g.tri_pm.data(), sizeof(int32_t) * g.tri_pm.size());
  return EFIE_OK;
}

int efie_rhs_planewave(efie_handle* h, int n_rhs, const double* khat, const double* pol, void* rhs,
                       void* stream) {
  if (!h) return EFIE_EINVAL;
  return guarded(h, [&] {
    if (n_rhs < 0 || !khat || !pol || (!rhs && n_rhs > 0)) throw EfieError{EFIE_EINVAL, "bad arguments"};
    if (n_rhs == 0) return EFIE_OK;
    cudaStream_t s = (cudaStream_t)stream;
    double* dk = h->mem.alloc<double>(3 * n_rhs);
    double* dp = h->mem.alloc<double>(3 * n_rhs);
    cuda_check(cudaMemcpyAsync(dk, khat, sizeof(double) * 3 * n_rhs, cudaMemcpyHostToDevice, s), "khat");
    cuda_check(cudaMemcpyAsync(dp, pol, sizeof(double) * 3 * n_rhs, cudaMemcpyHostToDevice, s), "pol");
    launch_rhs_planewave(h->dV, h->dT, h->darea, h->dtri_pm, h->dfree_pm, h->plan.g.N, h->plan.k, dk, dp, n_rhs,
                         (double2*)rhs, h->plan.g.N, s);
    cuda_check(cudaStreamSynchronize(s), "rhs");
    h->mem.release(dk);
    h->mem.release(dp);
    return EFIE_OK;
  });
}

int efie_matvec(efie_handle* h, const void* x, void* y, int n_rhs, void* stream) {
  if (!h) return EFIE_EINVAL;
  return guarded(h, [&] {
    if (n_rhs < 0 || ((!x || !y) && n_rhs > 0)) throw EfieError{EFIE_EINVAL, "bad arguments"};
    if (x == y && n_rhs > 0) throw EfieError{EFIE_EINVAL, "x and y must not alias"};
    if (n_rhs == 0) return EFIE_OK;
    do_matvec(h, (const double2*)x, h->plan.g.N, (double2*)y, nullptr, nullptr, h->plan.g.N, n_rhs, false,
              (cudaStream_t)stream);
    return EFIE_OK;
  });
}

int efie_matvec_host(efie_handle* h, const void* x_host, void* y_host, int n_rhs, void* stream) {
  if (!h) return EFIE_EINVAL;
  return guarded(h, [&] {
    if (n_rhs < 0 || ((!x_host || !y_host) && n_rhs > 0)) throw EfieError{EFIE_EINVAL, "bad arguments"};
    if (n_rhs == 0) return EFIE_OK;
    const int64_t N = h->plan.g.N;
    int Rc = h->opt.rhs_chunk > 0 ? std::min(h->opt.rhs_chunk, 8) : 8;
    // a slot holds a chunk pair when the top-level pass takes two chunks
    if (Rc == 8 && n_rhs >= 16 && pair_fits(h)) Rc = 16;
    HostPipe& hp = h->pipe;
    if (!hp.ready) {
      cuda_check(cudaStreamCreateWithFlags(&hp.s_in, cudaStreamNonBlocking), "host pipe stream");
      cuda_check(cudaStreamCreateWithFlags(&hp.s_out, cudaStreamNonBlocking), "host pipe stream");
      cuda_check(cudaEventCreateWithFlags(&hp.ev_start, cudaEventDisableTiming), "host pipe event");
      cuda_check(cudaEventCreateWithFlags(&hp.ev_end, cudaEventDisableTiming), "host pipe event");
      for (int b = 0; b < 2; ++b) {
        cuda_check(cudaEventCreateWithFlags(&hp.ev_in[b], cudaEventDisableTiming), "host pipe event");
        cuda_check(cudaEventCreateWithFlags(&hp.ev_comp[b], cudaEventDisableTiming), "host pipe event");
        cuda_check(cudaEventCreateWithFlags(&hp.ev_out[b], cudaEventDisableTiming), "host pipe event");
      }
      hp.ready = true;
    }
    if (hp.rc < Rc) {
      // the previous slots may still be in use by earlier calls
      cuda_check(cudaStreamSynchronize(hp.s_in), "host pipe");
      cuda_check(cudaStreamSynchronize(hp.s_out), "host pipe");
      for (int b = 0; b < 2; ++b) {
        if (hp.xs[b]) cuda_check(cudaEventSynchronize(hp.ev_comp[b]), "host pipe");
        h->mem.release(hp.xs[b]);
        h->mem.release(hp.ys[b]);
        hp.xs[b] = h->mem.alloc<double2>((int64_t)Rc * N);
        hp.ys[b] = h->mem.alloc<double2>((int64_t)Rc * N);
      }
      hp.rc = Rc;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const double2* xh = (const double2*)x_host;
    double2* yh = (double2*)y_host;
    // the copies start after the caller's earlier work on its stream
    cuda_check(cudaEventRecord(hp.ev_start, s), "host pipe");
    cuda_check(cudaStreamWaitEvent(hp.s_in, hp.ev_start, 0), "host pipe");
    cuda_check(cudaStreamWaitEvent(hp.s_out, hp.ev_start, 0), "host pipe");
    for (int i = 0, r0 = 0; r0 < n_rhs; ++i, r0 += Rc) {
      const int b = i & 1, nr = std::min(Rc, n_rhs - r0);
      const size_t bytes = sizeof(double2) * (size_t)nr * (size_t)N;
      // slot b's x is free once the product of two chunks back has run
      cuda_check(cudaStreamWaitEvent(hp.s_in, hp.ev_comp[b], 0), "host pipe");
      cuda_check(cudaMemcpyAsync(hp.xs[b], xh + (int64_t)r0 * N, bytes, cudaMemcpyHostToDevice, hp.s_in),
                 "host pipe H2D");
      cuda_check(cudaEventRecord(hp.ev_in[b], hp.s_in), "host pipe");
      // slot b's y is free once its copy-out of two chunks back has run
      cuda_check(cudaStreamWaitEvent(s, hp.ev_in[b], 0), "host pipe");
      cuda_check(cudaStreamWaitEvent(s, hp.ev_out[b], 0), "host pipe");
      do_matvec(h, hp.xs[b], N, hp.ys[b], nullptr, nullptr, N, nr, false, s);
      cuda_check(cudaEventRecord(hp.ev_comp[b], s), "host pipe");
      cuda_check(cudaStreamWaitEvent(hp.s_out, hp.ev_comp[b], 0), "host pipe");
      cuda_check(cudaMemcpyAsync(yh + (int64_t)r0 * N, hp.ys[b], bytes, cudaMemcpyDeviceToHost, hp.s_out),
                 "host pipe D2H");
      cuda_check(cudaEventRecord(hp.ev_out[b], hp.s_out), "host pipe");
    }
    cuda_check(cudaEventRecord(hp.ev_end, hp.s_out), "host pipe");
    cuda_check(cudaStreamWaitEvent(s, hp.ev_end, 0), "host pipe");
    return EFIE_OK;
  });
}

int efie_matvec_fp64(efie_handle* h, const void* x, void* y, int n_rhs, void* stream) {
  if (!h) return EFIE_EINVAL;
  return guarded(h, [&] {
    if (n_rhs < 0 || ((!x || !y) && n_rhs > 0)) throw EfieError{EFIE_EINVAL, "bad arguments"};
    if (x == y && n_rhs > 0) throw EfieError{EFIE_EINVAL, "x and y must not alias"};
    if (n_rhs == 0) return EFIE_OK;
    do_matvec(h, (const double2*)x, h->plan.g.N, (double2*)y, nullptr, nullptr, h->plan.g.N, n_rhs, true,
              (cudaStream_t)stream);
    return EFIE_OK;
  });
}

int efie_matvec_parts(efie_handle* h, const void* x, void* yA, void* yV, int n_rhs, void* stream) {
  if (!h) return EFIE_EINVAL;
  return guarded(h, [&] {
    if (n_rhs < 0 || (!x && n_rhs > 0)) throw EfieError{EFIE_EINVAL, "bad arguments"};
    if (n_rhs > 0 && (yA == x || yV == x || (yA && yA == yV)))
      throw EfieError{EFIE_EINVAL, "yA, yV and x must not alias"};
    if (n_rhs == 0) return EFIE_OK;
    do_matvec(h, (const double2*)x, h->plan.g.N, nullptr, (double2*)yA, (double2*)yV, h->plan.g.N, n_rhs,
              false, (cudaStream_t)stream);
    return EFIE_OK;
  });
}

int efie_solve(efie_handle* h, const void* rhs, void* x, int n_rhs, double tol, efie_solve_info* info,
               void* stream) {
  if (!h) return EFIE_EINVAL;
  return guarded(h, [&] {
    if (n_rhs < 0 || ((!rhs || !x) && n_rhs > 0)) throw EfieError{EFIE_EINVAL, "bad arguments"};
    if (rhs == x && n_rhs > 0) throw EfieError{EFIE_EINVAL, "rhs and x must not alias"};
    if (n_rhs == 0) return EFIE_OK;
    return solve_impl(h, (const double2*)rhs, (double2*)x, n_rhs, tol, info, (cudaStream_t)stream);
  });
}

int efie_profile(efie_handle* h, int enable) {
  if (!h) return EFIE_EINVAL;
  if (enable) h->prof.clear();
  h->prof.on = enable != 0;
  return EFIE_OK;
}

int efie_profile_read(efie_handle* h, int idx, char* name, int name_len, double* ms, int64_t* launches) {
  if (!h || idx < 0 || idx >= K_NCLASS) return EFIE_EINVAL;
  if (name && name_len > 0) {
    std::strncpy(name, kclass_name[idx], (size_t)name_len - 1);
    name[name_len - 1] = 0;
  }
  double tot = 0;
  for (auto& e : h->prof.ev) {
    if (e.first != idx) continue;
    if (cudaEventSynchronize(e.second.second) != cudaSuccess) return EFIE_ECUDA;
    float t = 0;
    cudaEventElapsedTime(&t, e.second.first, e.second.second);
    tot += t;
  }
  if (ms) *ms = tot;
  if (launches) *launches = h->prof.launches[idx];
  return EFIE_OK;
}

int efie_launch_count(const efie_handle* h, int64_t* n) {
  if (!h || !n) return EFIE_EINVAL;
  *n = h->n_launches;
  return EFIE_OK;
}

int efie_setup_times(const efie_handle* h, double* seconds, int n, int* n_phases) {
  if (!h || n < 0) return EFIE_EINVAL;
  for (int i = 0; i < std::min(n, 4); ++i)
    if (seconds) seconds[i] = h->setup_s[i];
  if (n_phases) *n_phases = 4;
  return EFIE_OK;
}

int efie_precond_harvest(efie_handle* h, const void* rhs, int n_rhs, int restart, int n_cycles, void* r_out,
                         void* e_out, void* stream) {
  if (!h) return EFIE_EINVAL;
  return guarded(h, [&] {
    if (n_rhs <= 0 || restart <= 0 || n_cycles <= 0 || !rhs || !r_out || !e_out)
      throw EfieError{EFIE_EINVAL, "bad arguments"};
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = h->plan.g.N;
    const double2* b = (const double2*)rhs;
    efie_options saved = h->opt;
    h->opt.precond = EFIE_PRECOND_NONE;
    // reference solution of the plain solver
    double2* xs = h->mem.alloc<double2>((int64_t)n_rhs * N);
    double2* rec = h->mem.alloc<double2>((int64_t)n_cycles * n_rhs * N);
    double2* tmp = h->mem.alloc<double2>((int64_t)n_rhs * N);
    h->opt.max_iters = std::max(saved.max_iters, 2000);
    solve_impl(h, b, xs, n_rhs, 1e-9, nullptr, s);
    // iterates of restarted GMRES(restart): x_j after cycle j
    h->opt.gmres_restart = restart;
    cuda_check(cudaMemsetAsync(rec, 0, sizeof(double2) * n_cycles * n_rhs * N, s), "rec");
    solve_impl(h, b, tmp, n_rhs, 1e-300, nullptr, s, rec, n_cycles);
    h->opt = saved;
    double2* ro = (double2*)r_out;
    double2* eo = (double2*)e_out;
    for (int c = 0; c < n_cycles; ++c) {
      double2* xc = rec + (int64_t)c * n_rhs * N;
      launch_lincomb(xs, xc, 1.0, -1.0, eo + (int64_t)c * n_rhs * N, (int64_t)n_rhs * N, s);
      do_matvec(h, xc, N, tmp, nullptr, nullptr, N, n_rhs, true, s);
      launch_lincomb(b, tmp, 1.0, -1.0, ro + (int64_t)c * n_rhs * N, (int64_t)n_rhs * N, s);
    }
    cuda_check(cudaStreamSynchronize(s), "harvest");
    h->mem.release(xs);
    h->mem.release(rec);
    h->mem.release(tmp);
    return EFIE_OK;
  });
}

int efie_precond_train(efie_handle* h, const void* r, const void* e, int n_pairs, int epochs, double lr,
                       uint64_t seed, int objective, double* loss_out, void* stream) {
  if (!h) return EFIE_EINVAL;
  return guarded(h, [&] {
    if (n_pairs <= 0 || epochs <= 0 || !(lr > 0) || !r || !e || objective < 0 || objective > 1)
      throw EfieError{EFIE_EINVAL, "bad arguments"};
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = h->plan.g.N;
    std::vector<float> p = h->net_params;
    if ((int)p.size() != efie::nn_param_count()) efie::nn_init_params(p, seed);
    net_activate(h, p, true);
    double2* z = h->mem.alloc<double2>(N);
    double2* g = h->mem.alloc<double2>(N);
    double2* w = h->mem.alloc<double2>(N);
    double2* t = h->mem.alloc<double2>(N);
    double* dn = h->mem.alloc<double>(2);
    std::mt19937_64 rng(seed);
    std::vector<int> order(n_pairs);
    const int batch = 4;
    for (int ep = 0; ep < epochs; ++ep) {
      for (int i = 0; i < n_pairs; ++i) order[i] = i;
      std::shuffle(order.begin(), order.end(), rng);
      double lsum = 0;
      for (int b0 = 0; b0 < n_pairs; b0 += batch) {
        const int nb = std::min(batch, n_pairs - b0);
        efie::nn_zero_grad(*h->net, s);
        for (int q = 0; q < nb; ++q) {
          const int i = order[b0 + q];
          const double2* ri = (const double2*)r + (int64_t)i * N;
          const double2* ei = (const double2*)e + (int64_t)i * N;
          efie::nn_forward(*h->net, ri, z, true, s);
          double num = 0, den = 1;
          if (objective == 0) {
            efie::nn_backward(*h->net, z, ei, g, s);
            cuda_check(cudaStreamSynchronize(s), "train");
            efie::nn_loss_terms(*h->net, &num, &den);
          } else {
            // L = |T z - r|^2 / |r|^2 ; dL/dz = 2 conj(T conj(T z - r)) / |r|^2 (T = T^T)
            do_matvec(h, z, N, w, nullptr, nullptr, N, 1, false, s);
            launch_lincomb(w, ri, 1.0, -1.0, w, N, s);
            launch_norms(w, N, N, 1, dn, s);
            launch_norms(ri, N, N, 1, dn + 1, s);
            double nn2[2];
            cuda_check(cudaMemcpyAsync(nn2, dn, sizeof(double) * 2, cudaMemcpyDeviceToHost, s), "d2h");
            cuda_check(cudaStreamSynchronize(s), "train");
            num = nn2[0];
            den = nn2[1];
            launch_conj_scale(w, 1.0, t, N, s);
            do_matvec(h, t, N, g, nullptr, nullptr, N, 1, false, s);
            launch_conj_scale(g, den > 0 ? 2.0 / den : 0.0, g, N, s);
            efie::nn_backward_g(*h->net, g, s);
          }
          lsum += den > 0 ? num / den : 0.0;
        }
        efie::nn_adam(*h->net, (float)lr, 1.0f / (float)nb, s);
      }
      if (loss_out) loss_out[ep] = lsum / n_pairs;
    }
    cuda_check(cudaStreamSynchronize(s), "train");
    efie::nn_read_params(*h->net, p);
    for (void* q : {(void*)z, (void*)g, (void*)w, (void*)t, (void*)dn}) h->mem.release(q);
    for (float v : p)
      if (!std::isfinite(v)) throw EfieError{EFIE_EINVAL, "training diverged (non-finite weights)"};
    net_activate(h, p, false);
    return EFIE_OK;
  });
}

int efie_precond_save(const efie_handle* h, const char* path) {
  if (!h || !path || h->net_params.empty()) return EFIE_EINVAL;
  FILE* f = std::fopen(path, "wb");
  if (!f) return EFIE_EINVAL;
  int32_t n = (int32_t)h->net_params.size();
  bool ok = std::fwrite("EFIENN01", 1, 8, f) == 8 && std::fwrite(&n, sizeof(n), 1, f) == 1 &&
            std::fwrite(h->net_params.data(), sizeof(float), n, f) == (size_t)n;
  std::fclose(f);
  return ok ? EFIE_OK : EFIE_EINVAL;
}

int efie_precond_load(efie_handle* h, const char* path) {
  if (!h || !path) return EFIE_EINVAL;
  return guarded(h, [&] {
    std::vector<float> w;
    if (!read_weights(path, w)) throw EfieError{EFIE_EINVAL, std::string("cannot read weights: ") + path};
    net_activate(h, w, false);
    h->opt.precond = EFIE_PRECOND_LEARNED;
    return EFIE_OK;
  });
}

int efie_precond_enable(efie_handle* h, int enable) {
  if (!h) return EFIE_EINVAL;
  h->opt.precond = enable ? EFIE_PRECOND_LEARNED : EFIE_PRECOND_NONE;
  return EFIE_OK;
}

int efie_precond_params(efie_handle* h, float* out, const float* in, int n) {
  if (!h || n != efie::nn_param_count()) return EFIE_EINVAL;
  return guarded(h, [&] {
    if (in) {
      std::vector<float> p(in, in + n);
      net_activate(h, p, false);
    }
    if (out) {
      if (h->net_params.empty()) throw EfieError{EFIE_EINVAL, "no network parameters"};
      std::memcpy(out, h->net_params.data(), sizeof(float) * n);
    }
    return EFIE_OK;
  });
}

int efie_precond_apply(efie_handle* h, const void* r, void* z, int n_vec, void* stream) {
  if (!h) return EFIE_EINVAL;
  return guarded(h, [&] {
    if (n_vec < 0 || ((!r || !z) && n_vec > 0)) throw EfieError{EFIE_EINVAL, "bad arguments"};
    if (r == z && n_vec > 0) throw EfieError{EFIE_EINVAL, "r and z must not alias"};
    if (!h->net) throw EfieError{EFIE_EINVAL, "no network loaded"};
    const int64_t N = h->plan.g.N;
    KScope ks(h, K_PRECOND, (cudaStream_t)stream, 6 * n_vec);
    for (int i = 0; i < n_vec; ++i)
      efie::nn_forward(*h->net, (const double2*)r + (int64_t)i * N, (double2*)z + (int64_t)i * N, false,
                       (cudaStream_t)stream);
    return EFIE_OK;
  });
}

int efie_precond_gradient(efie_handle* h, const void* r, const void* e, float* grad, double* loss, void* stream) {
  if (!h) return EFIE_EINVAL;
  return guarded(h, [&] {
    if (!r || !e) throw EfieError{EFIE_EINVAL, "bad arguments"};
    if (h->net_params.empty()) throw EfieError{EFIE_EINVAL, "no network parameters"};
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<float> p = h->net_params;
    net_activate(h, p, true);
    double2* z = h->mem.alloc<double2>(h->plan.g.N);
    double2* gb = h->mem.alloc<double2>(h->plan.g.N);
    efie::nn_zero_grad(*h->net, s);
    efie::nn_forward(*h->net, (const double2*)r, z, true, s);
    efie::nn_backward(*h->net, z, (const double2*)e, gb, s);
    cuda_check(cudaStreamSynchronize(s), "gradient");
    double num = 0, den = 1;
    efie::nn_loss_terms(*h->net, &num, &den);
    if (loss) *loss = num / den;
    std::vector<float> g;
    efie::nn_read_grads(*h->net, g);
    if (grad) std::memcpy(grad, g.data(), sizeof(float) * g.size());
    h->mem.release(z);
    h->mem.release(gb);
    net_activate(h, p, false);
    return EFIE_OK;
  });
}

int efie_autotune_set(efie_handle* h, int rhs_chunk, int mac_variant, int near_variant) {
  if (!h || rhs_chunk < 1 || rhs_chunk > 8 || mac_variant < 0 || mac_variant > 5 || near_variant < 0 ||
      near_variant > 3)
    return EFIE_EINVAL;
  h->opt.rhs_chunk = rhs_chunk;
  h->mac_variant = mac_variant;
  h->near_variant = near_variant;
  return EFIE_OK;
}

int efie_transform_schedule_set(efie_handle* h, int schedule) {
  if (!h || schedule < 0 || schedule > 3) return EFIE_EINVAL;
  h->fft_variant = schedule;
  return EFIE_OK;
}

int efie_transform_schedule_get(const efie_handle* h, int* schedule) {
  if (!h || !schedule) return EFIE_EINVAL;
  *schedule = h->fft_variant;
  return EFIE_OK;
}

int efie_autotune(efie_handle* h, int n_rhs, void* stream, int* best_chunk, int* best_mac, int* best_near) {
  if (!h) return EFIE_EINVAL;
  return guarded(h, [&] {
    if (n_rhs <= 0) throw EfieError{EFIE_EINVAL, "n_rhs must be positive"};
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = h->plan.g.N;
    double2* x = h->mem.alloc<double2>((int64_t)n_rhs * N);
    double2* y = h->mem.alloc<double2>((int64_t)n_rhs * N);
    cuda_check(cudaMemsetAsync(x, 0, sizeof(double2) * n_rhs * N, s), "x");
    const bool prof = h->prof.on;
    h->prof.on = false;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int bc = 8, bm = 0, bn = 0;
    for (int chunk : {8, 4, 2, 1}) {
      if (chunk > n_rhs && chunk != 1) continue;
      for (int cand = 0; cand < 24; ++cand) {
        const int mv = cand % 6, nv = cand / 6;
        if (nv > 0 && !h->near_df) continue;  // the near variants differ in the mixed form only
        if (mv == 4 && (chunk != 8 || n_rhs < 16)) continue;  // differs from 0 on chunk pairs only
        h->opt.rhs_chunk = chunk;
        h->mac_variant = mv;
        h->near_variant = nv;
        do_matvec(h, x, N, y, nullptr, nullptr, N, n_rhs, false, s);  // warm-up / allocation
        cudaEventRecord(e0, s);
        do_matvec(h, x, N, y, nullptr, nullptr, N, n_rhs, false, s);
        cudaEventRecord(e1, s);
        cuda_check(cudaEventSynchronize(e1), "autotune");
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
          best = ms;
          bc = chunk;
          bm = mv;
          bn = nv;
        }
      }
    }
    h->opt.rhs_chunk = bc;
    h->mac_variant = bm;
    h->near_variant = bn;
    // then the transform schedule with the chosen kernels (it differs only
    // for FP32 passes of 8 right-hand sides)
    if (h->precision == EFIE_MIXED && bc == 8) {
      float best_f = 1e30f;
      int bf = 0;
      for (int fv = 0; fv < 4; ++fv) {
        h->fft_variant = fv;
        do_matvec(h, x, N, y, nullptr, nullptr, N, n_rhs, false, s);
        cudaEventRecord(e0, s);
        do_matvec(h, x, N, y, nullptr, nullptr, N, n_rhs, false, s);
        cudaEventRecord(e1, s);
        cuda_check(cudaEventSynchronize(e1), "autotune");
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_f) {
          best_f = ms;
          bf = fv;
        }
      }
      h->fft_variant = bf;
    }
    h->prof.on = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->mem.release(x);
    h->mem.release(y);
    if (best_chunk) *best_chunk = bc;
    if (best_mac) *best_mac = bm;
    if (best_near) *best_near = bn;
    return EFIE_OK;
  });
}

int efie_destroy(efie_handle* h) {
  if (!h) return EFIE_EINVAL;
  delete h;
  return EFIE_OK;
}

}  // extern "C"

// ----------------------------------------------------------------- batches
struct efie_batch {
  std::vector<efie_handle*> hs;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  cudaEvent_t fork = nullptr;
  cudaStream_t cap = nullptr;   // capture stream (the caller's may be the legacy default stream)
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  std::vector<const void*> key_x;
  std::vector<void*> key_y;
  std::vector<int> key_n;
  int64_t launches = 0;
  std::string err;
  ~efie_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (auto st : streams) cudaStreamDestroy(st);
    for (auto ev : events) cudaEventDestroy(ev);
    if (fork) cudaEventDestroy(fork);
    if (cap) cudaStreamDestroy(cap);
  }
};

extern "C" {

int efie_batch_create(efie_handle* const* hs, int n, efie_batch** out) {
  if (!hs || n <= 0 || !out) return EFIE_EINVAL;
  efie_batch* b = new (std::nothrow) efie_batch();
  if (!b) return EFIE_ENOMEM;
  for (int i = 0; i < n; ++i) {
    if (!hs[i]) {
      delete b;
      return EFIE_EINVAL;
    }
    b->hs.push_back(hs[i]);
    cudaStream_t st;
    cudaEvent_t ev;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      delete b;
      return EFIE_ECUDA;
    }
    b->streams.push_back(st);
    b->events.push_back(ev);
  }
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
    delete b;
    return EFIE_ECUDA;
  }
  *out = b;
  return EFIE_OK;
}

// One CUDA-graph launch for the products of every member: member i computes
// y[i] = T_i x[i] for n_rhs[i] vectors, on its own branch of the graph.
int efie_batch_matvec(efie_batch* b, const void* const* x, void* const* y, const int* n_rhs, void* stream) {
  if (!b || !x || !y || !n_rhs) return EFIE_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = b->hs.size();
  std::vector<const void*> kx(x, x + n);
  std::vector<void*> ky(y, y + n);
  std::vector<int> kn(n_rhs, n_rhs + n);
  try {
    // every member's arguments before any member's work
    for (size_t i = 0; i < n; ++i)
      if (kn[i] < 0 || (kn[i] > 0 && (!x[i] || !y[i] || x[i] == y[i])))
        throw EfieError{EFIE_EINVAL, "bad batch arguments (member " + std::to_string(i) + ")"};
    if (!b->exec || kx != b->key_x || ky != b->key_y || kn != b->key_n) {
      // allocate every member's buffers outside the capture
      for (size_t i = 0; i < n; ++i) {
        efie_handle* h = b->hs[i];
        if (kn[i] > 0)
          do_matvec(h, (const double2*)x[i], h->plan.g.N, (double2*)y[i], nullptr, nullptr, h->plan.g.N, kn[i],
                    false, s);
      }
      cuda_check(cudaStreamSynchronize(s), "batch warm-up");
      if (b->exec) cudaGraphExecDestroy(b->exec);
      if (b->graph) cudaGraphDestroy(b->graph);
      b->exec = nullptr;
      b->graph = nullptr;
      std::vector<bool> prof(n);
      for (size_t i = 0; i < n; ++i) {
        prof[i] = b->hs[i]->prof.on;
        b->hs[i]->prof.on = false;
      }
      cudaStream_t c = b->cap;
      cuda_check(cudaStreamBeginCapture(c, cudaStreamCaptureModeThreadLocal), "capture");
      cuda_check(cudaEventRecord(b->fork, c), "fork");
      for (size_t i = 0; i < n; ++i) {
        efie_handle* h = b->hs[i];
        cuda_check(cudaStreamWaitEvent(b->streams[i], b->fork, 0), "fork wait");
        if (kn[i] > 0)
          do_matvec(h, (const double2*)x[i], h->plan.g.N, (double2*)y[i], nullptr, nullptr, h->plan.g.N, kn[i],
                    false, b->streams[i]);
        cuda_check(cudaEventRecord(b->events[i], b->streams[i]), "join");
        cuda_check(cudaStreamWaitEvent(c, b->events[i], 0), "join wait");
      }
      cuda_check(cudaStreamEndCapture(c, &b->graph), "end capture");
      for (size_t i = 0; i < n; ++i) b->hs[i]->prof.on = prof[i];
      cuda_check(cudaGraphInstantiate(&b->exec, b->graph, 0), "instantiate");
      b->key_x = kx;
      b->key_y = ky;
      b->key_n = kn;
    }
    cuda_check(cudaGraphLaunch(b->exec, s), "graph launch");
    b->launches++;
    return EFIE_OK;
  } catch (const EfieError& e) {
    cudaGraph_t g = nullptr;
    cudaStreamCaptureStatus st;
    if (cudaStreamIsCapturing(b->cap, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
      cudaStreamEndCapture(b->cap, &g);
      if (g) cudaGraphDestroy(g);
    }
    b->err = e.msg;
    g_last_error = e.msg;
    return e.code;
  }
}

int efie_batch_destroy(efie_batch* b) {
  if (!b) return EFIE_EINVAL;
  delete b;
  return EFIE_OK;
}

const char* efie_last_error(const efie_handle* h) {
  if (h) return h->err.c_str();
  return g_last_error.c_str();
}

}  // extern "C"
