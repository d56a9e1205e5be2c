// Device-side data descriptors and kernel launchers shared by the CUDA
// translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace efie {

// Near field (always FP64).  Block j of the CSR near lists couples target box
// blk_tgt[j] with source box near_src[j]; A blocks are [n_rwg(x)][n_rwg(y)],
// V blocks [n_tri(x)][n_tri(y)], column-major ([col][row]), in sorted basis
// order.
struct NearDev {
  const double* V;          // [nv][3]
  const int32_t* T;         // [nt][3]
  const double* area;       // [nt]
  double k;
  int64_t n_boxes, n_blocks;
  const int64_t* near_ptr;  // [B+1]
  const int32_t* near_src;  // [n_blocks]
  const int32_t* blk_tgt;   // [n_blocks]
  const int64_t* blkA_off;  // [n_blocks+1]
  const int64_t* blkV_off;  // [n_blocks+1]
  const int64_t* box_rwg_ptr;
  const int64_t* box_tri_ptr;
  const int32_t* tri_perm;  // sorted -> canonical triangle
  const int64_t* tset_ptr;
  const int32_t* tset;
  const int32_t* rwg_tl;
  const int32_t* rwg_loc;
  const double* rwg_coef;
  double2* A;               // [nnzA]
  double2* Vn;              // [nnzV]
  const int32_t* tri_tl;    // [nt sorted] index of the triangle in the tset of its own box, -1 if absent
  // direct factorization (Sec. VI-B): the scalar part on the RWG pairs of the
  // A blocks, Phi[i][n] = int int div f_i div f_n g (same layout as A), or null
  double2* Phi;
};
// Blocks (x, y) with x > y are not integrated: T is symmetric, so they are the
// transposes of the (y, x) blocks, copied by launch_near_mirror.

int near_upload_rules(const double* q3, const double* q4);
void launch_near_pairs_A(const NearDev& nd, int64_t j0, int64_t nblk, const int64_t* scr_off,
                         double2* scratch, int64_t total, cudaStream_t s);
void launch_near_combine_A(const NearDev& nd, int64_t j0, int64_t nblk, const int64_t* scr_off,
                           const double2* scratch, int64_t e_begin, int64_t total, cudaStream_t s);
// V entries of the blocks j in [j0, j0 + nblk) (entries [e_begin, e_begin + total)),
// reading I0 from the A pass's pair scratch of the same blocks where both
// triangles are in the A triangle sets, computing it otherwise.
void launch_near_V_pairs(const NearDev& nd, int64_t j0, int64_t nblk, const int64_t* scr_off,
                         const double2* scratch, int64_t e_begin, int64_t total, cudaStream_t s);
// M[blk] = M[mirror]^T for the n listed blocks (column-major blocks; box_ptr:
// the per-box function ranges that size them).
void launch_near_mirror(double2* M, const int64_t* blk_off, const int64_t* box_ptr, const int32_t* blk_tgt,
                        const int32_t* near_src, const int64_t* mir_blk, const int64_t* mir_src, int64_t n,
                        cudaStream_t s);
void launch_near_spmv(const double2* M, const int64_t* blk_off, const int64_t* near_ptr,
                      const int32_t* near_src, const int64_t* box_ptr, int64_t n_boxes,
                      const double2* x, double2* y, int64_t ld, int nr, cudaStream_t s);

void launch_split_df(double2* a, int64_t n, cudaStream_t s);
void launch_split_vec(const double2* x, float4* y, int64_t n, cudaStream_t s);
void launch_near_spmv_df(const float4* M, const int64_t* blk_off, const int64_t* near_ptr,
                         const int32_t* near_src, const int64_t* box_ptr, int64_t n_boxes, const float4* x,
                         double2* y, int64_t ld, int nr, int variant, int* err, cudaStream_t s);

// Strided tensor view of a box-batched 3D grid with channels innermost:
// element (b, i0, i1, i2, c) at b*sb + i0*s0 + i1*s1 + i2*s2 + c.
struct View {
  int64_t sb, s0, s1, s2;
};

template <typename R>
void launch_mode(const cpx_t<R>* in, View vin, cpx_t<R>* out, View vout, int64_t B, int C, int ax,
                 int nin, int e0, int e1, int e2, const void* M0, const void* M1, bool complex_m,
                 const int8_t* sel, const int64_t* srcmap, bool accumulate, cudaStream_t s);

// one pass of the sibling-shared upward transfer: out[g] = M(bit0) in[src0] +
// M(bit1) in[src1] along axis ax (src1 < 0: absent; src0 < 0: an output
// without inputs, written as zeros), M(0) = M0, M(1) = M1; nin (the child
// level's splines per axis) at most TRANSFER_MAX_SPLINES
constexpr int TRANSFER_MAX_SPLINES = 40;
template <typename R>
void launch_mode_pair(const cpx_t<R>* in, View vin, cpx_t<R>* out, View vout, int64_t G, int C, int ax, int nin,
                      int e0, int e1, int e2, const R* M0, const R* M1, const int64_t* src0, const int64_t* src1,
                      const int8_t* bit0, const int8_t* bit1, cudaStream_t s);

// DFT passes of the stabilized transforms using the conjugate symmetry of
// M = F P (forward, n x nin) / P^T F^{-1} (inverse, nout x n); false when no
// specialisation fits
template <typename R>
bool launch_dft(const cpx_t<R>* in, View vin, cpx_t<R>* out, View vout, int64_t B, int C, int ax, int nin,
                int e0, int e1, int e2, const cpx_t<R>* M, int n, bool inverse, cudaStream_t s);
// fused second and third transform passes, FP32, 32 channels, on (box,
// x-frequency) slabs; false when they do not apply
bool launch_dft_yz(const float2* in, float2* out, int64_t B, int sp, int n, const float2* M, bool inverse,
                   cudaStream_t s);
bool dft_yz_fits(int sp, int n);   // the fused forward pass takes this level
bool dft_zy_fits(int sp, int n);   // the fused inverse pass takes this level


// DFT passes of the stabilized transforms using the conjugate symmetry of
// M = F P (forward, n x nin) / P^T F^{-1} (inverse, nout x n); false when no
// specialisation fits
template <typename R>
bool launch_dft(const cpx_t<R>* in, View vin, cpx_t<R>* out, View vout, int64_t B, int C, int ax, int nin,
                int e0, int e1, int e2, const cpx_t<R>* M, int n, bool inverse, cudaStream_t s);

// top grid level on the tensor cores (tcgen05, kind::tf32 with a 3-term split,
// FP32-class products); false when the configuration does not fit it
bool mac_top_tc_fits(int C, int max_tile_targets, int64_t O);
// persistent warp-specialised form, on nch = 1 or 2 chunks of 8 right-hand
// sides per pass; tiles of <= 128 targets with any source lists; nq = sum over
// tiles of ceil(sources / 16)
bool mac_top_tc2_fits(int C, int max_tile_targets, int64_t O, int64_t nq, int64_t ntiles, int nch);
bool launch_mac_top_tc2(const float2* const* Qh, float2* const* Rh, int nch, const float2* Kh, int64_t B, int C,
                        int64_t O, int64_t nf, int64_t ntiles, int max_tile_targets, const int64_t* tgt_ptr,
                        const int32_t* tgt, const int64_t* src_ptr, const int32_t* src, const int64_t* kidx_off,
                        const int16_t* kidx, int64_t nq, int* err, cudaStream_t s);
// the same contract, fed by a loader warp (TMA bulk copies of index blocks,
// source spectra and kernel rows into shared-memory stages)
bool mac_top_tc3_fits(int C, int max_tile_targets, int64_t O, int64_t nq, int64_t ntiles, int nch);
bool launch_mac_top_tc3(const float2* const* Qh, float2* const* Rh, int nch, const float2* Kh, int64_t B, int C,
                        int64_t O, int64_t nf, int64_t ntiles, int max_tile_targets, const int64_t* tgt_ptr,
                        const int32_t* tgt, const int64_t* src_ptr, const int32_t* src, const int64_t* kidx_off,
                        const int32_t* kidx, int64_t nq, int* err, cudaStream_t s);
bool launch_mac_top_tc(const float2* Qh, float2* Rh, const float2* Kh, int64_t B, int C, int64_t O, int64_t nf,
                       int64_t ntiles, int max_tile_targets, const int64_t* tgt_ptr, const int32_t* tgt,
                       const int64_t* src_ptr, const int32_t* src, const int64_t* kidx_off, const int32_t* kidx,
                       int* err, cudaStream_t s);

template <typename R>
void launch_gather_build(const R* mr, const int32_t* mr_base, const int32_t* mr_ext, const int64_t* mr_off,
                         const R* mt, const int32_t* mt_base, const int32_t* mt_ext, const int64_t* mt_off,
                         const int64_t* box_rwg_ptr, const int64_t* box_tri_ptr, int64_t B, int sp,
                         int32_t* gptr_r, int32_t* gptr_t, R* gr, R* gt, cudaStream_t s);

// out_box: grid box of each of the B leaves (null: leaf b writes box b)
template <typename R>
void launch_anterp(const R* gr, const R* gt, const int32_t* gptr_r, const int32_t* gptr_t, const int64_t* mr_off,
                   const int64_t* mt_off, const int64_t* box_rwg_ptr, const int64_t* box_tri_ptr, int64_t B,
                   const int32_t* out_box, const cpx_t<R>* xs, int64_t ldx, const cpx_t<R>* rho, int64_t ldr, int nr,
                   cpx_t<R>* q, int sp, cudaStream_t s);

template <typename R>
void launch_interp(const R* mr, const int32_t* mr_base, const int32_t* mr_ext, const int64_t* mr_off,
                   const int32_t* rwg_box, int64_t N, const R* mt, const int32_t* mt_base,
                   const int32_t* mt_ext, const int64_t* mt_off, const int32_t* tri_box, int64_t Nt,
                   const cpx_t<R>* r, int sp, int nr, double2* yA, int64_t ldy, double2* u,
                   int64_t ldu, cudaStream_t s);

template <typename R>
void launch_mac(const cpx_t<R>* Qh, cpx_t<R>* Rh, const cpx_t<R>* Kh, int64_t B, int C, int64_t O,
                int64_t nf, int64_t ntiles, int max_tile_targets, const int64_t* tgt_ptr, const int32_t* tgt,
                const int64_t* src_ptr, const int32_t* src, const int64_t* kidx_off, const int32_t* kidx,
                cudaStream_t s);


// the six Hessian kernel spectra of the dyadic factorization (ab = 00, 01,
// 02, 11, 12, 22), [n^3][O] each
template <typename R>
struct KH6 {
  const cpx_t<R>* k[6];
};
// R[x][a] = sum_{y in IL(x)} sum_b H_ab(x - y) Q[y][b] for the three vector
// components (Sec. VI-C), fourth component zero; Q, R [n^3][B][4 nr]
template <typename R>
void launch_mac_dyad(const cpx_t<R>* Q, cpx_t<R>* Rout, KH6<R> K, int64_t B, int nr, int64_t nf, int64_t O,
                     const int64_t* il_ptr, const int32_t* il_src, const int32_t* il_off, cudaStream_t s);
void launch_kernel_samples(double2* Kc, const int32_t* offsets, int64_t o0, int64_t no, int n,
                           int shat, double h, double Delta, double k, int comp, cudaStream_t s);
template <typename R>
void launch_convert(const double2* in, cpx_t<R>* out, int64_t n, cudaStream_t s);

// misc vector kernels (FP64, c128)
void launch_permute_in(const double2* x, int64_t ldx, const int32_t* perm, int64_t N, int nr,
                       double2* xs, cudaStream_t s);
void launch_charges(const double2* xs, int64_t ldx, const int32_t* tri_rwg, const int8_t* tri_sgn,
                    int64_t Nt, int nr, double2* rho, int64_t ldr, cudaStream_t s);
void launch_combine(const double2* yA, int64_t ldA, const double2* w, int64_t ldw, const double2* yAn,
                    const double2* wn, const int32_t* rwg_perm, const int32_t* rwg_tri_sorted, int64_t N, int nr,
                    double2 cA, double2 cV, double2* y, int64_t ldy, double2* yAout,
                    double2* yVout, cudaStream_t s);
void launch_rhs_planewave(const double* V, const int32_t* T, const double* area, const int32_t* tri_pm,
                          const int32_t* free_pm, int64_t N, double k, const double* khat,
                          const double* pol, int nr, double2* rhs, int64_t ld, cudaStream_t s);

// Krylov helpers (FP64)
void launch_multidot(const double2* Vb, int64_t ldv_r, int64_t ldv_i, int nbasis, const double2* w,
                     int64_t ldw, int64_t N, int nr, const int* active, double2* h, cudaStream_t s);
void launch_multiaxpy(const double2* Vb, int64_t ldv_r, int64_t ldv_i, int nbasis, const double2* h,
                      int hstride, double2* w, int64_t ldw, int64_t N, int nr, const int* active,
                      double sign, cudaStream_t s);
void launch_lincomb(const double2* x, const double2* y, double a, double b, double2* out, int64_t n,
                    cudaStream_t s);
void launch_conj_scale(const double2* x, double a, double2* out, int64_t n, cudaStream_t s);
void launch_norms(const double2* w, int64_t ldw, int64_t N, int nr, double* out, cudaStream_t s);

}  // namespace efie
