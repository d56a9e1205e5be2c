// Host-side planning for the stabilized multilevel B-spline fast EFIE.
// Everything here runs once in efie_setup / efie_plan, in FP64 on the host:
// RWG geometry (Sec. II), the uniform octree and per-level spline parameters
// (Sec. III-B, IV-C, IV-D), knot insertion, stabilization and projector
// matrices (Sec. IV-B, V-B, Table I), exact moments (Eq. TAfactor, Sec. VI-A),
// interaction lists and the block structure of the near field.
#pragma once
#include <array>
#include <complex>
#include <cstdint>
#include <string>
#include <vector>

namespace efie {

using cplx = std::complex<double>;

struct EfieError {
  int code;
  std::string msg;
};

struct Geometry {
  int64_t nv = 0, nt = 0, N = 0;
  std::vector<double> V;            // [nv][3]
  std::vector<int32_t> T;           // [nt][3]
  std::vector<int32_t> edge;        // [N][2] (lo, hi)
  std::vector<int32_t> tri_pm;      // [N][2] (c+, c-)
  std::vector<int32_t> free_pm;     // [N][2] vertex ids of x+, x-
  std::vector<double> area;         // [nt]
  std::vector<double> cen;          // [nt][3]
};

struct Level {
  int level = 0;
  int s = 0, sb = 0, sp = 0, shat = 0, nfft = 0;
  double h = 0, delta = 0, Delta = 0;
  std::vector<int64_t> ijk;          // [B][3] occupied boxes, Morton order
  std::vector<uint64_t> code;        // [B] Morton codes (sorted)
  std::vector<int64_t> parent;       // [B] index at level-1 (grid levels above top: -1)
  std::vector<int64_t> child_ptr;    // [B+1] children (level+1) of each box
  // interaction list (CSR over target boxes)
  std::vector<int64_t> il_ptr;       // [B+1]
  std::vector<int32_t> il_src;       // [nnz] source box
  std::vector<int32_t> il_off;       // [nnz] offset id
  std::vector<int32_t> offsets;      // [O][3] o = ijk_target - ijk_source
  std::vector<uint8_t> leaf;         // [B] 1 for a leaf of the tree (its functions are anterpolated here)
  // translation tiles: groups of <= TILE_T targets sharing one source list;
  // kidx[tile] is [n_src][TILE_T] offset ids (-1: pair not translated here)
  std::vector<int64_t> tile_tgt_ptr, tile_src_ptr, tile_kidx_off;
  std::vector<int32_t> tile_tgt, tile_src, tile_kidx;
  // tensor-core tiles of an interaction-list level: TILE_TOP consecutive
  // boxes as targets, the union of their interaction lists as sources (sorted),
  // and the offset id of every (source, target) slot, -1 outside the lists
  std::vector<int64_t> tct_tgt_ptr, tct_src_ptr, tct_kidx_off;
  std::vector<int32_t> tct_tgt, tct_src, tct_kidx;
  // dense per-level matrices (row-major, FP64)
  std::vector<double> P;             // [shat][sp] = B_stab^-1 S
  std::vector<double> CL, CR;        // [sp_parent][sp_this] (child = this level)
  std::vector<cplx> Mf;              // [nfft][sp] = F[:, :shat] P
  std::vector<cplx> Mb;              // [sp][nfft] = P^T Finv[:shat, :]
  std::vector<cplx> Fn;              // [nfft][nfft] full DFT (kernel spectra)
};

struct MomentBlocks {
  // per basis function (sorted order): base index and extents of its dense
  // block in the leaf box grid, offset of its data; data is [ncomp][e0][e1][e2]
  std::vector<int32_t> base;   // [n][3]
  std::vector<int32_t> ext;    // [n][3]
  std::vector<int64_t> off;    // [n+1]
  std::vector<double> data;
};

constexpr int TILE_X = 8;      // targets per thread in the translation MAC
constexpr int TILE_TOP = 128;  // targets per tile on the top grid level

struct Plan {
  Geometry g;
  double k = 0;
  int p = 0, D = 0, top = 0, n_levels = 0;
  double root_lo[3] = {0, 0, 0}, root_edge = 0;
  std::vector<Level> lv;             // lv[ell - top], ell = top..D
  Level& L(int ell) { return lv[ell - top]; }
  const Level& L(int ell) const { return lv[ell - top]; }

  // leaves: the boxes of level D (uniform tree), or the leaves of every level
  // (nonuniform tree, Sec. VII), numbered level by level from the top level,
  // Morton order within a level.  The near field's boxes are these leaves.
  bool adaptive = false;
  int64_t n_leaves = 0;
  std::vector<int32_t> leaf_level;      // [NL]
  std::vector<int64_t> leaf_box;        // [NL] box index on its level
  std::vector<int64_t> level_leaf_ptr;  // [n_levels+1]: leaves of level top+i are [ptr[i], ptr[i+1])

  // basis-function ordering (sorted by leaf)
  std::vector<int32_t> rwg_perm;     // sorted k -> canonical m
  std::vector<int32_t> rwg_box;      // sorted k -> leaf
  std::vector<int64_t> box_rwg_ptr;  // [NL+1]
  std::vector<int32_t> tri_perm;     // sorted t -> canonical triangle
  std::vector<int32_t> tri_box;      // sorted t -> leaf
  std::vector<int64_t> box_tri_ptr;  // [NL+1]
  std::vector<int32_t> rwg_lbox, tri_lbox;  // sorted function -> box index on its leaf's level
  std::vector<int32_t> tri_rank;     // canonical triangle -> sorted index
  std::vector<int32_t> rwg_tri_sorted;  // [N_sorted][2] sorted triangle index of c+, c-

  // near field structure over the leaves (uniform: leaf boxes with
  // |d|_inf <= 1; nonuniform: ancestors on the coarser level adjacent or equal)
  std::vector<int64_t> near_ptr;     // [NL+1]
  std::vector<int32_t> near_src;     // source box
  std::vector<int64_t> blkA_off;     // [nnz_blocks+1] offset of A block (entries)
  std::vector<int64_t> blkV_off;     // [nnz_blocks+1]
  int64_t nnzA = 0, nnzV = 0;
  // triangle set per leaf box for A assembly: triangles of RWGs in the box
  std::vector<int64_t> tset_ptr;     // [NL+1]
  std::vector<int32_t> tset;         // canonical triangle ids
  std::vector<int32_t> rwg_tl;       // [N_sorted][2] local index in tset of its box
  std::vector<int32_t> rwg_loc;      // [N_sorted][2] local vertex index of the free vertex
  std::vector<double> rwg_coef;      // [N_sorted][2] sigma / (2 a)

  MomentBlocks mom_rwg;              // 3 components
  MomentBlocks mom_tri;              // 1 component (pulse, includes 1/a)
  MomentBlocks mom_div;              // 1 component, RWG divergence (+-1/a on c+-), RWG blocks; only
                                     // when built with_div (direct factorization, Sec. VI-B)
};

// Builds everything except moments when with_moments is false; with_div adds
// the RWG divergence moments of the direct factorization.
void build_plan(Plan& P, const double* xyz, int64_t nv, const int32_t* tri, int64_t nt,
                double k, int p, double grid_spacing, int levels, int n_splines,
                bool with_moments, bool with_div = false);

// ------------------------------------------------------------ nonuniform tree
// Sec. VII: a box is subdivided while it holds more than max_elems triangles
// (by centroid), unless a basis function would then protrude from its child
// box by more than max_prot of the child's edge.  Per-level s and s_b follow
// Sec. IV-C/D with the buffer rule for leaves on the parent level.
struct AdaptiveOptions {
  int max_elems = 200;
  double max_prot = 0.25;
  int top = 2;          // top grid level; leaves above it are rejected
  int n_splines = 0;    // s on the deepest level; 0 -> p + 4
  int max_depth = 30;
};

struct AdaptiveLevel {
  int level = 0, s = 0, sb = 0, sp = 0, shat = 0;
  double h = 0, delta = 0;
  std::vector<std::array<int64_t, 3>> key;  // boxes, sorted
  std::vector<uint8_t> leaf;                // per box
  std::vector<int32_t> n_rwg, n_tri;        // functions whose leaf is the box
  std::vector<int64_t> parent;              // index on level - 1 (-1 on the top level)
  std::vector<int64_t> child_ptr, child;    // children on level + 1 (CSR)
  int64_t n_far_pairs = 0;                  // translated box pairs on this level
  int64_t n_leaf_rwg = 0, n_leaf_tri = 0;
};

struct AdaptivePlan {
  Geometry g;
  double root_lo[3] = {0, 0, 0}, root_edge = 0;
  int D = 0, top = 0, p = 0;
  std::vector<AdaptiveLevel> lv;            // lv[ell - top]
  std::vector<int32_t> rwg_level, rwg_box, tri_level, tri_box;   // canonical function -> its leaf
  // leaves of all levels, numbered level by level from the top, boxes in key order
  std::vector<int32_t> leaf_level;
  std::vector<int64_t> leaf_box;            // index of the leaf on its level
  // functions sorted by leaf (then canonical id): sorted -> canonical, sorted -> leaf
  std::vector<int32_t> rwg_perm, rwg_leaf, tri_perm, tri_leaf, tri_rank;
  std::vector<int64_t> leaf_rwg_ptr, leaf_tri_ptr;
  // near leaves (CSR over leaves, sources ascending): leaves whose ancestors on
  // the coarser of their two levels are adjacent or equal
  std::vector<int64_t> near_ptr;
  std::vector<int32_t> near_src;
  // ordered pairs of functions whose leaves are near (self pairs included)
  int64_t near_pairs_rwg = 0, near_pairs_tri = 0;
  // exact moments in each function's leaf (with_moments), sorted order
  MomentBlocks mom_rwg, mom_tri;
};

void build_adaptive_plan(AdaptivePlan& A, const double* xyz, int64_t nv, const int32_t* tri, int64_t nt,
                         double k, int p, const AdaptiveOptions& o, bool with_moments = false);

// The nonuniform tree as a plan of the device pipeline (boxes in Morton order,
// leaves of every level as the near field's boxes, moments in each function's
// own leaf); with_div as in build_plan.
void build_plan_adaptive(Plan& P, const double* xyz, int64_t nv, const int32_t* tri, int64_t nt, double k, int p,
                         const AdaptiveOptions& o, bool with_moments, bool with_div = false);

// Spline helpers exposed for tests of the host code
std::vector<double> open_knots(double lo, double hi, int ns, int p);
std::vector<double> restriction_matrix(const std::vector<double>& Up,
                                       const std::vector<double>& Uc, int p, int* rows,
                                       int* cols);
void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w);

}  // namespace efie
