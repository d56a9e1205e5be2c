/*
 * efie.h -- C ABI of the GB300 stabilized multilevel B-spline fast EFIE library.
 *
 * The library solves the discretized PEC electric field integral equation
 *     T j = e,   T = jk A + (jk)^-1 Sigma V Sigma^T
 * (Sec. II, Eq. discretizedEFIE, with the star form of Sec. VI-A), where A is
 * the Galerkin vector-potential matrix of RWG functions without edge-length
 * normalization (Eq. matTA), V the single-layer matrix of pulse functions
 * phi_c = 1/a_c and Sigma the star matrix.  Products with T use the fast
 * method of Sec. III-V: exact B-spline moments, knot-insertion interlevel
 * transfers, knot-removal stabilization (Table I), FFT-accelerated Toeplitz
 * translations per level, and a sparse FP64 near-field correction.
 *
 * Conventions shared by every call:
 *  - SI units: metres, wavenumber k in rad/m; time dependence e^{j w t}.
 *  - Unknown m is the RWG of the m-th mesh edge in lexicographic order of its
 *    (lower, higher) vertex ids; its c+ triangle is the one whose
 *    counter-clockwise vertex cycle runs lower -> higher.
 *  - Complex vectors are interleaved (re, im) doubles ("c128"), laid out
 *    [n_rhs][N] row-major, in device memory owned by the caller unless a call
 *    says otherwise.  Calls enqueue work on the caller's CUDA stream `stream`
 *    (a cudaStream_t passed as void*, NULL = legacy default stream).
 *  - Return codes: 0 success, negative error, positive EFIE_NOT_CONVERGED.
 *    efie_last_error() gives a message for the last failure of the handle.
 *
 * Every call that computes runs in this library's CUDA kernels on the current
 * device; there is no CPU fallback.  A call made without a usable CUDA device
 * returns EFIE_ECUDA.
 */
#ifndef EFIE_GB300_H
#define EFIE_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EFIE_OK 0
#define EFIE_EINVAL (-1)        /* bad mesh, parameter or size */
#define EFIE_ENOMEM (-2)        /* device or host allocation failed / over limit */
#define EFIE_ECUDA (-3)         /* CUDA runtime error or no device */
#define EFIE_ETIMEOUT (-4)      /* a bounded device wait expired */
#define EFIE_NOT_CONVERGED 1    /* solver stopped at max_iters; x holds the best iterate */

#define EFIE_FP64 0             /* plain form: every step in complex FP64 */
#define EFIE_MIXED 1            /* far field in complex FP32; near field, projector
                                   construction, Arnoldi and true residual in FP64 */

#define EFIE_FACT_STAR 0        /* star-based factorization (Sec. VI-A): RWG moments for the
                                   vector part, pulse moments of the charges for the scalar
                                   part, near A on RWG pairs and V on triangle pairs */
#define EFIE_FACT_DIRECT 1      /* direct factorization (Sec. VI-B): RWG and RWG-divergence
                                   moments in the RWG's leaf box, one near set of RWG pairs
                                   holding A and Phi = Sigma V Sigma^T */
#define EFIE_FACT_DYADIC 2      /* dyadic factorization (Sec. VI-C): the three RWG moment
                                   components translated with g and with the Hessian of g
                                   (the scalar part is -int int f_m . grad grad g . f_n), near
                                   field as in the direct form */

#define EFIE_PRECOND_NONE 0
#define EFIE_PRECOND_LEARNED 1  /* learned mesh-local FGMRES preconditioner (not in
                                   the paper); falls back to NONE when unusable */

typedef struct efie_handle efie_handle;   /* opaque, library-owned */

/* Closed, consistently oriented triangle mesh (outward CCW).  Caller-owned host
 * arrays, copied by efie_setup. */
typedef struct {
    int64_t n_vertices;
    const double *xyz;      /* [n_vertices][3] metres */
    int64_t n_triangles;
    const int32_t *tri;     /* [n_triangles][3] vertex ids */
} efie_mesh;

typedef struct {
    int32_t n_splines;       /* leaf splines per axis s; 0 -> p + 4 (Sec. VII-B) */
    int32_t precision;       /* EFIE_FP64 or EFIE_MIXED */
    int32_t gmres_restart;   /* 0 -> 100 */
    int32_t max_iters;       /* 0 -> 1000 */
    int32_t precond;         /* EFIE_PRECOND_* */
    int32_t rhs_chunk;       /* right-hand sides per far-field pass; 0 -> automatic */
    const char *weights_path;/* learned preconditioner weights, or NULL */
    int64_t device_mem_limit;/* bytes; 0 -> no limit beyond the device */
    uint64_t seed;
    int32_t factorization;   /* EFIE_FACT_STAR (default), EFIE_FACT_DIRECT or EFIE_FACT_DYADIC */
} efie_options;

/* Per-level summary filled by efie_plan / efie_level_info. */
typedef struct {
    int32_t level;           /* octree level (root 0) */
    int32_t s, sb, sp, shat; /* splines, buffer splines, s' = s + 2 sb, stabilized count */
    int32_t nfft;            /* FFT length per axis (>= 2 shat - 1) */
    int64_t n_boxes;         /* occupied boxes */
    int64_t n_far_pairs;     /* translated box pairs at this level */
    int64_t n_offsets;       /* distinct translation offsets (kernel spectra) */
    double h, delta, Delta;  /* box edge, knot spacing, interpolation-point spacing */
} efie_level_info_t;

typedef struct {
    int64_t n_unknowns, n_triangles;
    int32_t depth, top_level, n_levels, p;
    double root_lo[3], root_edge;
    int64_t near_nnz_A, near_nnz_V;  /* near entries of A and of the scalar part (V on triangle
                                       pairs; Phi on A's RWG pairs for a direct-factorization
                                       handle) */
    int64_t device_bytes;    /* estimated resident device bytes of the setup products */
    int64_t moment_entries_rwg;  /* leaf moment entries of all RWGs, per vector component */
    int64_t moment_entries_tri;  /* leaf moment entries of the scalar part: triangles (star),
                                    RWG divergences (direct handle) */
} efie_plan_info_t;

typedef struct {
    int32_t iterations;          /* matvecs spent on this right-hand side */
    double true_rel_residual;    /* ||e - T x|| / ||e|| with the FP64 fast matvec */
    int32_t converged;           /* 1 if true_rel_residual <= tol */
    int32_t precond_fallback;    /* 1 if the learned preconditioner was dropped */
} efie_solve_info;

/* Host-only planning (no device work): octree, per-level spline parameters and
 * interaction counts for the problem efie_setup would build (Sec. III-B, IV-C,
 * IV-D, Table I).  levels_out may be NULL; otherwise it must hold
 * max_levels entries.  Returns EFIE_EINVAL for a bad mesh or parameters (p not
 * in 1..6, levels outside 1..depth+1, grid spacing so small that the buffer
 * splines close the gap between far interpolation domains). */
int efie_plan(const efie_mesh *mesh, double wavenumber, int spline_degree,
              double grid_spacing, int levels, const efie_options *opt,
              efie_plan_info_t *info, efie_level_info_t *levels_out, int max_levels);

/* Nonuniform octree (Sec. VII): a box is subdivided while it holds more than
 * max_elems triangles (by centroid), unless a basis function would then
 * protrude from its child box by more than max_prot of the child's edge. */
typedef struct {
    int32_t max_elems;       /* the paper uses 200 */
    double max_prot;         /* the paper uses 0.25 */
    int32_t top;             /* top grid level (root 0), >= 1; leaves above it are rejected */
    int32_t n_splines;       /* s on the deepest level; 0 -> p + 4 */
    int32_t max_depth;       /* 0 -> 30 */
} efie_tree_options;

/* Per-level summary of a nonuniform tree (efie_plan_adaptive). */
typedef struct {
    int32_t level;           /* octree level (root 0) */
    int32_t s, sb, sp, shat; /* splines, buffer splines, s' = s + 2 sb, stabilized count */
    int64_t n_boxes;         /* boxes on the level (leaves and parents) */
    int64_t n_leaves;
    int64_t n_far_pairs;     /* translated box pairs on this level */
    int64_t n_leaf_rwg, n_leaf_tri;  /* functions whose leaf is on this level */
    double h, delta;         /* box edge, knot spacing */
} efie_adaptive_level_t;

/* Host-only planning of a nonuniform octree (Sec. VII tree rule; per-level s
 * and s_b by Sec. IV-C/D, with the buffer rule for leaves on the parent
 * level).  Every basis function belongs to the leaf holding its point (edge
 * midpoint, centroid); level l translates the non-adjacent box pairs with
 * adjacent parents (every non-adjacent pair on the top level); two leaves are
 * near when, on the coarser of their levels, their ancestors are adjacent or
 * equal.  levels_out (may be NULL) receives min(max_levels, n_levels) levels
 * from the top level down; *n_levels the level count; *near_pairs_rwg and
 * *near_pairs_tri the ordered pairs of RWGs / triangles in near leaves (self
 * pairs included).  Any output pointer may be NULL.  topt NULL -> the paper's
 * values (200, 0.25, top 2).  EFIE_EINVAL for a bad mesh or parameters, a
 * leaf above the top level, or buffer splines that close the gap between far
 * interpolation domains.  efie_setup_adaptive sets up the device pipeline on
 * the same tree. */
int efie_plan_adaptive(const efie_mesh *mesh, double wavenumber, int spline_degree,
                       const efie_tree_options *topt, efie_adaptive_level_t *levels_out, int max_levels,
                       int32_t *n_levels, int64_t *near_pairs_rwg, int64_t *near_pairs_tri);

/* Host-only: the leaves and near-leaf lists of the nonuniform tree of
 * efie_plan_adaptive.  Leaves are numbered level by level from the top level,
 * boxes in (i, j, k) order: leaf_level [n_leaves], leaf_ijk [n_leaves][3];
 * near_ptr [n_leaves + 1] and near_src [nnz] (CSR, sources ascending) list,
 * for each leaf, the leaves whose ancestors on the coarser of the two levels
 * are adjacent or equal.  Call with the arrays NULL to get *n_leaves and
 * *nnz; each array must then hold that many entries: leaf_cap >= n_leaves
 * for leaf_level and leaf_ijk, leaf_cap >= n_leaves + 1 when near_ptr is
 * given (it is sized by leaf_cap too), near_cap >= nnz; else EFIE_EINVAL.  Other errors as efie_plan_adaptive. */
int efie_plan_adaptive_near(const efie_mesh *mesh, double wavenumber, int spline_degree,
                            const efie_tree_options *topt, int64_t *n_leaves, int64_t *nnz,
                            int32_t *leaf_level, int64_t *leaf_ijk, int64_t leaf_cap,
                            int64_t *near_ptr, int32_t *near_src, int64_t near_cap);

/* Host-only: exact moments of the nonuniform tree, each function in its
 * own leaf's splines (that level's s', knots and buffers), as
 * efie_setup_adaptive uploads them.  kind 0: RWGs
 * (canonical edge ids), [3][sp][sp][sp] per id; kind 1: triangles, pulse
 * 1/area, [sp][sp][sp] per id.  The blocks are packed one after the other in
 * out (out_len entries), each with its own sp; level_out and sp_out (n_ids
 * entries each, may be NULL) return the leaf level and sp of every id.  Call
 * with out NULL to get the needed length in *out_needed.  EFIE_EINVAL for a
 * bad kind or id or a short buffer; other errors as efie_plan_adaptive. */
int efie_plan_adaptive_moments(const efie_mesh *mesh, double wavenumber, int spline_degree,
                               const efie_tree_options *topt, int kind, const int32_t *ids, int64_t n_ids,
                               double *out, int64_t out_len, int64_t *out_needed, int32_t *level_out,
                               int32_t *sp_out);

/* Host-only: the per-level dense matrices of the far pipeline, row-major FP64.
 *   P[level]   (shat x sp)   = B_stab^{-1} S (Sec. V-B)
 *   CL, CR     (sp_parent x sp_child) interlevel transfers into level-1 (Sec. IV-B)
 * `which`: 0 = P, 1 = C^L, 2 = C^R.  `out` must hold rows*cols doubles; rows
 * and cols are returned.  For C^L/C^R, `level` is the child level. */
int efie_plan_matrix(const efie_mesh *mesh, double wavenumber, int spline_degree,
                     double grid_spacing, int levels, const efie_options *opt,
                     int level, int which, double *out, int64_t out_len,
                     int32_t *rows, int32_t *cols);

/* Host-only: the exact moments of the leaf splines (Eq. TAfactor,
 * Sec. VI-A) that efie_setup uploads, for a list of basis functions.
 *   kind 0: RWG edges (canonical edge index, the order of efie_rwg_edges),
 *           out[i][d][a][b][c] = integral over the RWG support of f_m,d N_abc;
 *   kind 1: triangles (canonical index), pulse 1/area:
 *           out[i][a][b][c] = integral over the triangle of N_abc / area;
 *   kind 2: RWG edges, divergence moments of the direct factorization
 *           (Sec. VI-B) in the RWG's leaf box:
 *           out[i][a][b][c] = integral over the RWG support of (div f_m) N_abc,
 *           div f_m = +-1/area on c+-.
 * a, b, c run over the sp splines per axis of the basis function's leaf box
 * (sp = s + 2 s_b); entries outside the function's support are 0.  out must
 * hold n_ids * (3 for kind 0, else 1) * sp^3 doubles (out_len); *sp_out returns sp.
 * EFIE_EINVAL for a bad mesh, parameters, kind or index, or a short buffer. */
int efie_plan_moments(const efie_mesh *mesh, double wavenumber, int spline_degree,
                      double grid_spacing, int levels, const efie_options *opt,
                      int kind, const int32_t *ids, int64_t n_ids, double *out,
                      int64_t out_len, int32_t *sp_out);

/* Build every setup product on the current device: geometry, octree,
 * transfers, projectors, exact moments, kernel spectra per level and
 * offset, and the FP64 near field (Sec. VI-A: RWG pairs for A and triangle
 * pairs for V, each in adjacent leaf boxes).  With opt->factorization =
 * EFIE_FACT_DIRECT (Sec. VI-B) the scalar part is anterpolated from the
 * divergence moments of every RWG in its own leaf box and interpolated back
 * onto them, and its near field Phi = Sigma V Sigma^T is assembled on the
 * RWG pairs of A's blocks (from the same triangle-pair integrals); products,
 * solves and the (A x, Phi x) split of efie_matvec_parts follow.  EFIE_EINVAL
 * also for a plan with more than 40 splines per axis on a level below the top
 * grid level (the interlevel transfer kernels take at most that).  With
 * EFIE_FACT_DYADIC (Sec. VI-C) the near field and moments are the direct
 * form's, and the far scalar part comes instead from the three RWG moment
 * components translated with the six entries of the Hessian of g (one more
 * set of kernel spectra per entry and offset, and a second output grid per
 * level); efie_matvec_parts returns (A x, -H x) with H the Hessian product
 * plus Phi on the near pairs.  Both precisions; the mixed form's far field
 * runs one chunk of right-hand sides at a time on CUDA cores.  opt may be
 * NULL (defaults).  EFIE_EINVAL for an unknown factorization.  On success
 * *out owns all device memory until efie_destroy. */
int efie_setup(const efie_mesh *mesh, double wavenumber, int spline_degree,
               double grid_spacing, int levels, const efie_options *opt,
               efie_handle **out);

/* efie_setup on the nonuniform octree of efie_plan_adaptive (Sec. VII tree
 * rule, topt NULL -> the paper's values): every level's grids take the
 * anterpolation of the functions whose leaves lie on it (each in its own
 * leaf's splines) before the upward transfer to the parent level, the
 * translations of the level's interaction lists, and after the downward
 * transfer the interpolation onto those functions; the near field holds the
 * RWG (A) and triangle (V) pairs of near leaves, leaves of different levels
 * included.  Everything else (precisions, products, solves, batching of
 * right-hand sides) as with efie_setup, in the star factorization (Sec. VI-A;
 * EFIE_EINVAL for another opt->factorization); the spline count of the
 * deepest level is topt->n_splines (opt->n_splines is not used).  Errors as
 * efie_setup and efie_plan_adaptive. */
int efie_setup_adaptive(const efie_mesh *mesh, double wavenumber, int spline_degree,
                        const efie_tree_options *topt, const efie_options *opt, efie_handle **out);

int efie_num_unknowns(const efie_handle *h, int64_t *n);
int efie_plan_info(const efie_handle *h, efie_plan_info_t *info);

/* Host arrays filled per unknown: edge_vertices [N][2] (lower, higher) and
 * tri_pm [N][2] (c+, c-). Either may be NULL. */
int efie_rwg_edges(const efie_handle *h, int32_t *edge_vertices, int32_t *tri_pm);

/* Plane-wave right-hand sides [e^i]_m = int f_m . pol_r exp(-jk khat_r . x) dS
 * (Sec. II), FP64.  khat, pol: host [n_rhs][3]; rhs: device c128 [n_rhs][N]. */
int efie_rhs_planewave(efie_handle *h, int n_rhs, const double *khat, const double *pol,
                       void *rhs, void *stream);

/* Same result as efie_rhs_planewave, for callers that must not allocate
 * device memory once running (a no-allocation or memory-pool policy, loops
 * that cannot take the synchronisation of cudaMalloc/cudaFree, hosts whose
 * allocator belongs to another framework).  It calls no cudaMalloc, cudaFree
 * or allocating library routine: khat and pol are staged in a fixed device
 * array of the library (4096 plane waves, 192 KiB), which every GPU that loads
 * the library keeps until the process exits.  n_rhs above 4096 returns
 * EFIE_EINVAL.  The paper has no counterpart; this is a deployment variant.
 * Notes: the handle's device must be current (else EFIE_EINVAL); the first
 * call on a device looks up that array's device address
 * (cudaGetSymbolAddress) with the device current, so make it before any
 * stream capture, and the address it keeps is valid until that device is
 * reset; all calls on a device share the array, so calls whose
 * copies and kernels overlap on the GPU race -- serialise them; the call
 * synchronises `stream` before returning. */
int efie_rhs_planewave_noalloc(efie_handle *h, int n_rhs, const double *khat, const double *pol,
                               void *rhs, void *stream);

/* y = T x for n_rhs vectors (device c128 [n_rhs][N]; x and y must not alias).
 * Uses the handle's precision.  Charges, anterpolation, upward
 * transfers, stabilized FFT translations, downward transfers, interpolation,
 * near field. */
int efie_matvec(efie_handle *h, const void *x, void *y, int n_rhs, void *stream);

/* y = T x with x and y in HOST memory (c128 [n_rhs][N]), the same product as
 * efie_matvec.  The right-hand sides go through the device in chunks of the
 * handle's chunk size (16 when two chunks of 8 share a top-level pass),
 * double-buffered: the copy-in of one chunk and the
 * copy-out of the previous one overlap the product of the current one, on two
 * copy streams of the handle, ordered after the caller's earlier work on
 * `stream`.  The call returns once the work is queued; y is complete when
 * `stream` has been synchronized.  x and y should be page-locked (pinned) for
 * the copies to overlap; pageable memory gives the same result without
 * overlap.  The handle keeps 2 x 2 staging buffers of chunk x N entries from
 * the first call until efie_destroy.  Calls on one handle must not overlap. */
int efie_matvec_host(efie_handle *h, const void *x_host, void *y_host, int n_rhs, void *stream);

/* Same product computed in FP64 regardless of the handle's precision (the
 * plain FP64 form used for true residuals).  Needs FP64 setup products, which
 * EFIE_MIXED handles keep alongside the FP32 ones. */
int efie_matvec_fp64(efie_handle *h, const void *x, void *y, int n_rhs, void *stream);

/* Separate parts, y_A = A x and y_V = Sigma V Sigma^T x (far + near), so that
 * T x = jk y_A + (jk)^-1 y_V.  Either output may be NULL; neither may alias x
 * or the other (EFIE_EINVAL). */
int efie_matvec_parts(efie_handle *h, const void *x, void *yA, void *yV, int n_rhs,
                      void *stream);

/* Solve T x = rhs by GMRES(m) (FGMRES with the learned preconditioner), x0 = 0,
 * FP64 CGS2 Arnoldi; success when the true relative residual, recomputed with
 * the FP64 fast matvec, is <= tol.  rhs, x: device c128 [n_rhs][N]; info: host
 * array of n_rhs entries or NULL.  Returns EFIE_NOT_CONVERGED if any rhs did not
 * reach tol within max_iters (x then holds the best iterate).  EFIE_EINVAL for
 * tol <= 0 or for x aliasing rhs (x0 = 0 would overwrite it). */
int efie_solve(efie_handle *h, const void *rhs, void *x, int n_rhs, double tol,
               efie_solve_info *info, void *stream);

/* ---- Learned preconditioner (not part of the paper) ----------------------
 * A message-passing network on the RWG adjacency graph (3 layers, width 64,
 * bfloat16 weights, FP32 accumulation on the tensor cores) maps a residual to
 * an approximate error and serves as the flexible right preconditioner of
 * FGMRES when enabled; a non-finite output switches that right-hand side back
 * to plain GMRES (efie_solve_info.precond_fallback = 1).  Weights files start
 * with the 8 bytes "EFIENN01", an int32 count, then float32 parameters. */

/* Residual/error pairs from the plain solver's own runs: e_j = x* - x_j and
 * r_j = rhs - T x_j for the iterates x_j of restarted GMRES(restart) after
 * cycles j = 0..n_cycles-1, x* a converged (1e-9) solution.  rhs: device c128
 * [n_rhs][N]; r_out, e_out: device c128 [n_cycles][n_rhs][N]. */
int efie_precond_harvest(efie_handle *h, const void *rhs, int n_rhs, int restart, int n_cycles,
                         void *r_out, void *e_out, void *stream);

/* Train (Adam, batches of 4 pairs) on n_pairs device pairs r, e (c128
 * [n_pairs][N]) for `epochs` passes.  objective 0 minimises the error loss
 * |net(r) - e|^2 / |e|^2; objective 1 the residual loss |T net(r) - r|^2 / |r|^2
 * (T e = r), whose gradient 2 conj(T conj(T z - r)) / |r|^2 costs two fast
 * matvecs per pair.  Starts from the handle's current weights (or a seeded
 * initialisation).  loss_out: host array of `epochs` mean losses, or NULL. */
int efie_precond_train(efie_handle *h, const void *r, const void *e, int n_pairs, int epochs, double lr,
                       uint64_t seed, int objective, double *loss_out, void *stream);
int efie_precond_save(const efie_handle *h, const char *path);
int efie_precond_load(efie_handle *h, const char *path);   /* also enables it */
int efie_precond_enable(efie_handle *h, int enable);
/* Copy the parameters out (out != NULL) and/or replace them (in != NULL); n must
 * equal the network's parameter count. */
int efie_precond_params(efie_handle *h, float *out, const float *in, int n);
/* z_i = net(r_i) for n_vec device c128 vectors [n_vec][N]; z must not alias r
 * (EFIE_EINVAL). */
int efie_precond_apply(efie_handle *h, const void *r, void *z, int n_vec, void *stream);
/* Loss and parameter gradient (host float[n]) of one pair at the current weights. */
int efie_precond_gradient(efie_handle *h, const void *r, const void *e, float *grad, double *loss,
                          void *stream);

/* ---- Batching over right-hand sides and meshes ----------------------------
 * efie_autotune times one product of n_rhs vectors for each candidate
 * right-hand-side chunk (8, 4, 2, 1 vectors per far-field pass), each
 * translation kernel choice (0: tensor cores, tcgen05 with a 3-term TF32
 * split of every FP32 operand, in the persistent warp-specialised form where
 * the level fits it and the far field is FP32, else as 3, else as 2; pairs
 * of 8-vector chunks also run the interaction-list levels below the top on
 * tensor cores; 1: register tiles; 2: CUDA cores with shared-memory staging
 * through the pair index tile; 3: tensor cores, one CTA per tile and
 * frequency; 4: as 0 with the interaction-list levels of chunk pairs on CUDA
 * cores; 5: as 0 with a persistent form whose loader warp stages index
 * blocks, source spectra and kernel rows in shared memory by asynchronous
 * copies) and, for
 * mixed handles, each near-field
 * kernel (0: source values staged in shared memory by double-buffered
 * asynchronous copies, one thread per row and 8 right-hand sides; 1: read
 * through L1 with no barriers; 2: staged by the block between barriers, 4
 * right-hand sides per thread; 3: as 0 with the staging in an mbarrier ring
 * filled by a copy warp, so that row warps never wait on one another), and
 * keeps the fastest in the handle; the
 * choices are returned if the pointers are set. */
int efie_autotune(efie_handle *h, int n_rhs, void *stream, int *best_chunk, int *best_mac, int *best_near);
/* Sets the three choices efie_autotune makes: rhs_chunk in 1..8, mac_variant
 * in 0..5 and near_variant in 0..3 as above.  EFIE_EINVAL outside those
 * ranges. */
int efie_autotune_set(efie_handle *h, int rhs_chunk, int mac_variant, int near_variant);
/* Transform schedule of the stabilized forward / inverse transforms
 * (Sec. III-C, V-B: the per-axis products with F P and P^T F^-1 on every
 * level).  0: three line passes per transform; 1: for FP32 passes of 8
 * right-hand sides (32 channels) and 9, 13 or 21 splines per axis, the
 * forward y and z passes run fused on (box, x-frequency) slabs in shared
 * memory, so the intermediate of the second pass never goes to device
 * memory; 2: the inverse z and y passes fused the same way as well; 3
 * (default): forward and inverse fused on levels of 9 splines per axis only,
 * line passes on the others.  All give the same operator up to rounding.
 * efie_autotune times all four (after choosing the other knobs) for mixed
 * handles whose best chunk is 8.  set: EFIE_EINVAL for a schedule outside
 * 0..3; get writes the handle's. */
int efie_transform_schedule_set(efie_handle *h, int schedule);
int efie_transform_schedule_get(const efie_handle *h, int *schedule);

/* A batch groups set-up handles (meshes of any size, same device).  Each
 * efie_batch_matvec runs y[i] = T_i x[i] (n_rhs[i] vectors, device c128) for
 * every member as ONE CUDA graph launch on `stream` (any stream, the legacy
 * default one included: capture uses an internal stream), each member on its
 * own branch of the graph.  The graph is captured on the first call and re-captured
 * whenever the pointers or counts change (that call also runs the products
 * once uncaptured to allocate the members' work buffers).  EFIE_EINVAL,
 * before any member's work, for a negative count, or for a member with vectors
 * whose x is NULL, y is NULL or y aliases x. */
typedef struct efie_batch efie_batch;
int efie_batch_create(efie_handle *const *hs, int n, efie_batch **out);
int efie_batch_matvec(efie_batch *b, const void *const *x, void *const *y, const int *n_rhs, void *stream);
int efie_batch_destroy(efie_batch *b);

/* Kernel-class timing for measurement.  efie_profile(h, 1) clears and starts
 * recording: every later call that launches kernels records a CUDA event pair
 * on the caller's stream around each class of kernels (anterpolation,
 * transfers, transforms, translation, interpolation, near field, vectors, ...);
 * efie_profile(h, 0) stops.  efie_profile_read synchronizes the recorded
 * events and returns, for class index idx (0-based, EFIE_EINVAL past the last),
 * its name (NUL-terminated, truncated to name_len), total milliseconds and
 * number of kernel launches.  Either output pointer may be NULL.  While
 * recording, a product runs its near field and its far field one after the
 * other (they overlap on two streams otherwise), so that each class's time is
 * its own kernels' time. */
int efie_profile(efie_handle *h, int enable);
int efie_profile_read(efie_handle *h, int idx, char *name, int name_len, double *ms,
                      int64_t *launches);

/* Number of this library's kernel launches issued through h since setup
 * (setup kernels excluded). */
int efie_launch_count(const efie_handle *h, int64_t *n);

/* Wall-clock seconds of the phases of efie_setup for h, in this order:
 * 0 host plan (geometry, octree, transfers, projectors, exact moments),
 * 1 device tables (uploads, transfer groups, translation tiles),
 * 2 near field (FP64 assembly of A and V, and the double-float split),
 * 3 far field (gather lists, kernel spectra, per-precision products).
 * Writes min(n, 4) values to seconds and the phase count to *n_phases (either
 * pointer may be NULL).  Host memory only; no device work. */
int efie_setup_times(const efie_handle *h, double *seconds, int n, int *n_phases);

int efie_destroy(efie_handle *h);

/* Message of the last error of h, or of the last failed setup/plan of this
 * thread when h is NULL.  Never NULL; valid until the next call. */
const char *efie_last_error(const efie_handle *h);

#ifdef __cplusplus
}
#endif
#endif /* EFIE_GB300_H */
