"""GB300-native stabilized multilevel B-spline fast EFIE (Python binding).

A thin ctypes layer over the C ABI declared in include/efie.h.  It only
marshals arguments: device vectors are torch tensors (complex128, CUDA) whose
data pointers and current CUDA stream are passed to the library, and every step
of the computation runs in the library's CUDA kernels.  Loading fails loudly if
the shared library has not been built (see ``build.py``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = ["load_library", "Options", "EFIE", "Batch", "plan", "plan_matrix", "EfieError",
           "EFIE_FP64", "EFIE_MIXED", "EFIE_PRECOND_NONE", "EFIE_PRECOND_LEARNED", "EFIE_FACT_STAR",
           "EFIE_FACT_DIRECT", "EFIE_FACT_DYADIC",
           "EXPORTED_SYMBOLS"]

EFIE_OK, EFIE_EINVAL, EFIE_ENOMEM, EFIE_ECUDA, EFIE_ETIMEOUT, EFIE_NOT_CONVERGED = 0, -1, -2, -3, -4, 1
EFIE_FP64, EFIE_MIXED = 0, 1
EFIE_PRECOND_NONE, EFIE_PRECOND_LEARNED = 0, 1
EFIE_FACT_STAR, EFIE_FACT_DIRECT, EFIE_FACT_DYADIC = 0, 1, 2

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libefie_gb300.so")

EXPORTED_SYMBOLS = [
    "efie_plan", "efie_plan_adaptive", "efie_plan_adaptive_near", "efie_plan_adaptive_moments", "efie_plan_matrix", "efie_plan_moments", "efie_setup", "efie_setup_adaptive", "efie_num_unknowns", "efie_plan_info",
    "efie_rwg_edges", "efie_rhs_planewave", "efie_rhs_planewave_noalloc", "efie_matvec", "efie_matvec_host",
    "efie_matvec_fp64",
    "efie_matvec_parts", "efie_solve", "efie_precond_harvest", "efie_precond_train", "efie_precond_save",
    "efie_precond_load", "efie_precond_enable", "efie_precond_params", "efie_precond_apply",
    "efie_precond_gradient", "efie_autotune", "efie_autotune_set", "efie_transform_schedule_set",
    "efie_transform_schedule_get", "efie_batch_create", "efie_batch_matvec",
    "efie_batch_destroy",
    "efie_profile", "efie_profile_read", "efie_launch_count", "efie_setup_times",
    "efie_destroy", "efie_last_error",
]


class EfieError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class _Mesh(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int64), ("xyz", ctypes.POINTER(ctypes.c_double)),
                ("n_triangles", ctypes.c_int64), ("tri", ctypes.POINTER(ctypes.c_int32))]


class Options(ctypes.Structure):
    _fields_ = [("n_splines", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("gmres_restart", ctypes.c_int32), ("max_iters", ctypes.c_int32),
                ("precond", ctypes.c_int32), ("rhs_chunk", ctypes.c_int32),
                ("weights_path", ctypes.c_char_p), ("device_mem_limit", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("factorization", ctypes.c_int32)]


class LevelInfo(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int32), ("s", ctypes.c_int32), ("sb", ctypes.c_int32),
                ("sp", ctypes.c_int32), ("shat", ctypes.c_int32), ("nfft", ctypes.c_int32),
                ("n_boxes", ctypes.c_int64), ("n_far_pairs", ctypes.c_int64),
                ("n_offsets", ctypes.c_int64), ("h", ctypes.c_double), ("delta", ctypes.c_double),
                ("Delta", ctypes.c_double)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n_unknowns", ctypes.c_int64), ("n_triangles", ctypes.c_int64),
                ("depth", ctypes.c_int32), ("top_level", ctypes.c_int32),
                ("n_levels", ctypes.c_int32), ("p", ctypes.c_int32),
                ("root_lo", ctypes.c_double * 3), ("root_edge", ctypes.c_double),
                ("near_nnz_A", ctypes.c_int64), ("near_nnz_V", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("moment_entries_rwg", ctypes.c_int64),
                ("moment_entries_tri", ctypes.c_int64)]


class TreeOptions(ctypes.Structure):
    _fields_ = [("max_elems", ctypes.c_int32), ("max_prot", ctypes.c_double), ("top", ctypes.c_int32),
                ("n_splines", ctypes.c_int32), ("max_depth", ctypes.c_int32)]


class AdaptiveLevelInfo(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int32), ("s", ctypes.c_int32), ("sb", ctypes.c_int32),
                ("sp", ctypes.c_int32), ("shat", ctypes.c_int32), ("n_boxes", ctypes.c_int64),
                ("n_leaves", ctypes.c_int64), ("n_far_pairs", ctypes.c_int64),
                ("n_leaf_rwg", ctypes.c_int64), ("n_leaf_tri", ctypes.c_int64),
                ("h", ctypes.c_double), ("delta", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("true_rel_residual", ctypes.c_double),
                ("converged", ctypes.c_int32), ("precond_fallback", ctypes.c_int32)]


_lib = None


def load_library(path: str = LIB_PATH):
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run paper_2606_13482_gb300/build.py)")
    lib = ctypes.CDLL(path)
    P, I32, I64, D, VP = ctypes.POINTER, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
    lib.efie_plan.argtypes = [P(_Mesh), D, ctypes.c_int, D, ctypes.c_int, P(Options), P(PlanInfo),
                              P(LevelInfo), ctypes.c_int]
    lib.efie_plan_matrix.argtypes = [P(_Mesh), D, ctypes.c_int, D, ctypes.c_int, P(Options), ctypes.c_int,
                                     ctypes.c_int, P(D), I64, P(I32), P(I32)]
    lib.efie_plan_adaptive.argtypes = [P(_Mesh), D, ctypes.c_int, P(TreeOptions), P(AdaptiveLevelInfo),
                                       ctypes.c_int, P(I32), P(I64), P(I64)]
    lib.efie_plan_adaptive_near.argtypes = [P(_Mesh), D, ctypes.c_int, P(TreeOptions), P(I64), P(I64), P(I32),
                                            P(I64), I64, P(I64), P(I32), I64]
    lib.efie_plan_adaptive_moments.argtypes = [P(_Mesh), D, ctypes.c_int, P(TreeOptions), ctypes.c_int, P(I32),
                                               I64, P(D), I64, P(I64), P(I32), P(I32)]
    lib.efie_plan_moments.argtypes = [P(_Mesh), D, ctypes.c_int, D, ctypes.c_int, P(Options), ctypes.c_int,
                                      P(I32), I64, P(D), I64, P(I32)]
    lib.efie_setup.argtypes = [P(_Mesh), D, ctypes.c_int, D, ctypes.c_int, P(Options), P(VP)]
    lib.efie_setup_adaptive.argtypes = [P(_Mesh), D, ctypes.c_int, P(TreeOptions), P(Options), P(VP)]
    lib.efie_num_unknowns.argtypes = [VP, P(I64)]
    lib.efie_plan_info.argtypes = [VP, P(PlanInfo)]
    lib.efie_rwg_edges.argtypes = [VP, P(I32), P(I32)]
    lib.efie_rhs_planewave.argtypes = [VP, ctypes.c_int, P(D), P(D), VP, VP]
    lib.efie_rhs_planewave_noalloc.argtypes = [VP, ctypes.c_int, P(D), P(D), VP, VP]
    lib.efie_matvec.argtypes = [VP, VP, VP, ctypes.c_int, VP]
    lib.efie_matvec_host.argtypes = [VP, VP, VP, ctypes.c_int, VP]
    lib.efie_matvec_fp64.argtypes = [VP, VP, VP, ctypes.c_int, VP]
    lib.efie_matvec_parts.argtypes = [VP, VP, VP, VP, ctypes.c_int, VP]
    lib.efie_solve.argtypes = [VP, VP, VP, ctypes.c_int, D, P(SolveInfo), VP]
    F = ctypes.c_float
    lib.efie_precond_harvest.argtypes = [VP, VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, VP, VP, VP]
    lib.efie_precond_train.argtypes = [VP, VP, VP, ctypes.c_int, ctypes.c_int, D, ctypes.c_uint64, ctypes.c_int,
                                       P(D), VP]
    lib.efie_precond_save.argtypes = [VP, ctypes.c_char_p]
    lib.efie_precond_load.argtypes = [VP, ctypes.c_char_p]
    lib.efie_precond_enable.argtypes = [VP, ctypes.c_int]
    lib.efie_precond_params.argtypes = [VP, P(F), P(F), ctypes.c_int]
    lib.efie_precond_apply.argtypes = [VP, VP, VP, ctypes.c_int, VP]
    lib.efie_precond_gradient.argtypes = [VP, VP, VP, P(F), P(D), VP]
    lib.efie_autotune.argtypes = [VP, ctypes.c_int, VP, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int)]
    lib.efie_autotune_set.argtypes = [VP, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.efie_transform_schedule_set.argtypes = [VP, ctypes.c_int]
    lib.efie_transform_schedule_get.argtypes = [VP, P(ctypes.c_int)]
    lib.efie_batch_create.argtypes = [P(VP), ctypes.c_int, P(VP)]
    lib.efie_batch_matvec.argtypes = [VP, P(VP), P(VP), P(ctypes.c_int), VP]
    lib.efie_batch_destroy.argtypes = [VP]
    lib.efie_profile.argtypes = [VP, ctypes.c_int]
    lib.efie_profile_read.argtypes = [VP, ctypes.c_int, ctypes.c_char_p, ctypes.c_int, P(D), P(I64)]
    lib.efie_launch_count.argtypes = [VP, P(I64)]
    lib.efie_setup_times.argtypes = [VP, P(D), ctypes.c_int, P(ctypes.c_int)]
    lib.efie_destroy.argtypes = [VP]
    lib.efie_last_error.argtypes = [VP]
    lib.efie_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _mesh(V, T):
    V = np.ascontiguousarray(V, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.int32)
    m = _Mesh(V.shape[0], V.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), T.shape[0],
              T.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return m, (V, T)


def planewave_args(khat, pol, out_shape=None, n_unknowns=None):
    """Directions and polarisations as contiguous float64 [n, 3] arrays of the
    same n; with out_shape, also checks that the output is [n, n_unknowns].
    The C ABI takes no sizes for these arrays, so this is their only guard."""
    khat = np.ascontiguousarray(np.atleast_2d(khat), dtype=np.float64)
    pol = np.ascontiguousarray(np.atleast_2d(pol), dtype=np.float64)
    if khat.ndim != 2 or khat.shape[1] != 3 or pol.shape != khat.shape:
        raise ValueError(f"khat and pol must both be [n, 3] (got {khat.shape} and {pol.shape})")
    if out_shape is not None and tuple(out_shape) != (khat.shape[0], n_unknowns):
        raise ValueError(f"out must be [{khat.shape[0]}, {n_unknowns}] (got {list(out_shape)})")
    return khat, pol


def _check(lib, rc, h=None):
    if rc < 0:
        raise EfieError(rc, lib.efie_last_error(h).decode())
    return rc


class Batch:
    """Set-up handles whose products run as one CUDA graph launch."""

    def __init__(self, handles):
        self.lib = load_library()
        self.handles = list(handles)
        arr = (ctypes.c_void_p * len(self.handles))(*[h.h.value for h in self.handles])
        b = ctypes.c_void_p()
        _check(self.lib, self.lib.efie_batch_create(arr, len(self.handles), ctypes.byref(b)))
        self.b = b

    def matvec(self, xs, ys):
        """ys[i] = T_i xs[i]; xs[i] and ys[i] are contiguous complex128 CUDA
        tensors [n_i, N_i] of the same shape (N_i: member i's unknowns)."""
        import torch
        n = len(self.handles)
        if len(xs) != n or len(ys) != n:
            raise ValueError(f"expected {n} inputs and {n} outputs (got {len(xs)} and {len(ys)})")
        for i, (h, x, y) in enumerate(zip(self.handles, xs, ys)):
            if x.dim() != 2:
                raise ValueError(f"xs[{i}] must be [n, N] (got {list(x.shape)})")
            h._vec(x)
            h._vec(EFIE._same_rows(x, y, f"ys[{i}]"))
        X = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
        Y = (ctypes.c_void_p * n)(*[y.data_ptr() for y in ys])
        R = (ctypes.c_int * n)(*[x.shape[0] for x in xs])
        _check(self.lib, self.lib.efie_batch_matvec(self.b, X, Y, R,
                                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
        return ys

    def close(self):
        if getattr(self, "b", None):
            self.lib.efie_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plan(V, T, k, p, grid_spacing, levels, options: Options | None = None):
    """Host-only planning: (plan info dict, list of per-level dicts)."""
    lib = load_library()
    m, keep = _mesh(V, T)
    info = PlanInfo()
    lv = (LevelInfo * 32)()
    _check(lib, lib.efie_plan(ctypes.byref(m), k, p, grid_spacing, levels,
                              ctypes.byref(options) if options else None, ctypes.byref(info), lv, 32))
    d = {f: getattr(info, f) for f, _ in PlanInfo._fields_}
    d["root_lo"] = list(info.root_lo)
    levels_out = [{f: getattr(lv[i], f) for f, _ in LevelInfo._fields_} for i in range(info.n_levels)]
    return d, levels_out


def plan_adaptive(V, T, k, p, max_elems=200, max_prot=0.25, top=2, n_splines=0, max_depth=0):
    """Host-only planning of a nonuniform octree (efie_plan_adaptive):
    (per-level dicts from the top level down, near RWG pairs, near triangle pairs)."""
    lib = load_library()
    m, keep = _mesh(V, T)
    o = TreeOptions(max_elems, max_prot, top, n_splines, max_depth)
    lv = (AdaptiveLevelInfo * 64)()
    n, nr, nt = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib, lib.efie_plan_adaptive(ctypes.byref(m), k, p, ctypes.byref(o), lv, 64, ctypes.byref(n),
                                       ctypes.byref(nr), ctypes.byref(nt)))
    levels = [{f: getattr(lv[i], f) for f, _ in AdaptiveLevelInfo._fields_} for i in range(n.value)]
    return levels, nr.value, nt.value


def plan_adaptive_near(V, T, k, p, max_elems=200, max_prot=0.25, top=2, n_splines=0, max_depth=0):
    """Leaves of the nonuniform tree and their near-leaf lists
    (efie_plan_adaptive_near): (leaf_level [L], leaf_ijk [L,3], near_ptr [L+1], near_src)."""
    lib = load_library()
    m, keep = _mesh(V, T)
    o = TreeOptions(max_elems, max_prot, top, n_splines, max_depth)
    nl, nz = ctypes.c_int64(), ctypes.c_int64()
    _check(lib, lib.efie_plan_adaptive_near(ctypes.byref(m), k, p, ctypes.byref(o), ctypes.byref(nl),
                                            ctypes.byref(nz), None, None, 0, None, None, 0))
    cap = nl.value + 1                      # near_ptr holds n_leaves + 1 entries
    lvl = np.zeros(cap, np.int32)
    ijk = np.zeros((cap, 3), np.int64)
    ptr = np.zeros(cap, np.int64)
    src = np.zeros(max(nz.value, 1), np.int32)
    ip = lambda a, t: a.ctypes.data_as(ctypes.POINTER(t))
    _check(lib, lib.efie_plan_adaptive_near(ctypes.byref(m), k, p, ctypes.byref(o), None, None,
                                            ip(lvl, ctypes.c_int32), ip(ijk, ctypes.c_int64), cap,
                                            ip(ptr, ctypes.c_int64), ip(src, ctypes.c_int32), src.size))
    return lvl[:nl.value], ijk[:nl.value], ptr, src[:nz.value]


def plan_adaptive_moments(V, T, k, p, kind, ids, max_elems=200, max_prot=0.25, top=2, n_splines=0, max_depth=0):
    """Exact moments of the nonuniform tree, each function in its own leaf
    (efie_plan_adaptive_moments): a list of arrays, [3,sp,sp,sp] (kind 0) or
    [sp,sp,sp] (kind 1) with each leaf level's sp, and the leaf levels."""
    lib = load_library()
    m, keep = _mesh(V, T)
    o = TreeOptions(max_elems, max_prot, top, n_splines, max_depth)
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    ip = lambda a, t: a.ctypes.data_as(ctypes.POINTER(t))
    need = ctypes.c_int64()
    lvl = np.zeros(ids.size, np.int32)
    sps = np.zeros(ids.size, np.int32)
    _check(lib, lib.efie_plan_adaptive_moments(ctypes.byref(m), k, p, ctypes.byref(o), kind,
                                               ip(ids, ctypes.c_int32), ids.size, None, 0, ctypes.byref(need),
                                               ip(lvl, ctypes.c_int32), ip(sps, ctypes.c_int32)))
    out = np.zeros(max(need.value, 1))
    _check(lib, lib.efie_plan_adaptive_moments(ctypes.byref(m), k, p, ctypes.byref(o), kind,
                                               ip(ids, ctypes.c_int32), ids.size, ip(out, ctypes.c_double),
                                               out.size, None, None, None))
    blocks, pos = [], 0
    nc = 3 if kind == 0 else 1
    for s in sps:
        n = nc * int(s) ** 3
        blk = out[pos:pos + n]
        blocks.append(blk.reshape((3, s, s, s) if kind == 0 else (s, s, s)))
        pos += n
    return blocks, lvl


def plan_matrix(V, T, k, p, grid_spacing, levels, level, which, options: Options | None = None):
    lib = load_library()
    m, keep = _mesh(V, T)
    r, c = ctypes.c_int32(), ctypes.c_int32()
    _check(lib, lib.efie_plan_matrix(ctypes.byref(m), k, p, grid_spacing, levels,
                                     ctypes.byref(options) if options else None, level, which, None, 0,
                                     ctypes.byref(r), ctypes.byref(c)))
    out = np.zeros(r.value * c.value)
    _check(lib, lib.efie_plan_matrix(ctypes.byref(m), k, p, grid_spacing, levels,
                                     ctypes.byref(options) if options else None, level, which,
                                     out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), out.size,
                                     None, None))
    return out.reshape(r.value, c.value)


def plan_moments(V, T, k, p, grid_spacing, levels, kind, ids, options: Options | None = None):
    """Host-only exact moments of the leaf splines (efie_plan_moments):
    kind 0 -> [n, 3, sp, sp, sp] for canonical RWG ids, kind 1 -> [n, sp, sp, sp]
    for triangle ids, kind 2 -> [n, sp, sp, sp] RWG divergence moments (direct
    factorization), each in the function's leaf box."""
    lib = load_library()
    m, keep = _mesh(V, T)
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    sp = ctypes.c_int32()
    opt = ctypes.byref(options) if options else None
    _check(lib, lib.efie_plan_moments(ctypes.byref(m), k, p, grid_spacing, levels, opt, kind,
                                      ids.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ids.size, None, 0,
                                      ctypes.byref(sp)))
    s = sp.value
    ncomp = 3 if kind == 0 else 1
    out = np.zeros(ids.size * ncomp * s ** 3)
    _check(lib, lib.efie_plan_moments(ctypes.byref(m), k, p, grid_spacing, levels, opt, kind,
                                      ids.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ids.size,
                                      out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), out.size, None))
    return out.reshape((ids.size, 3, s, s, s) if kind == 0 else (ids.size, s, s, s))


class EFIE:
    """Handle to a set-up problem on the current CUDA device."""

    def __init__(self, V, T, k, p, grid_spacing=None, levels=None, precision=EFIE_FP64, tree=None, **opts):
        """Uniform octree of (grid_spacing, levels) (efie_setup), or with
        `tree` = dict(max_elems, max_prot, top, n_splines, max_depth) the
        nonuniform octree of Sec. VII (efie_setup_adaptive; grid_spacing and
        levels unused)."""
        if tree is None and (grid_spacing is None or levels is None):
            raise ValueError("grid_spacing and levels are needed without a tree")
        import torch  # noqa: F401  (device memory and streams)
        self.lib = load_library()
        o = Options()
        o.precision = precision
        for key, val in opts.items():
            setattr(o, key, val)
        self.options = o
        m, keep = _mesh(V, T)
        h = ctypes.c_void_p()
        if tree is None:
            _check(self.lib, self.lib.efie_setup(ctypes.byref(m), k, p, grid_spacing, levels, ctypes.byref(o),
                                                 ctypes.byref(h)))
        else:
            t = dict(max_elems=200, max_prot=0.25, top=2, n_splines=0, max_depth=0)
            unknown = set(tree) - set(t)
            if unknown:
                raise ValueError(f"unknown tree options: {sorted(unknown)}")
            t.update(tree)
            to = TreeOptions(t["max_elems"], t["max_prot"], t["top"], t["n_splines"], t["max_depth"])
            _check(self.lib, self.lib.efie_setup_adaptive(ctypes.byref(m), k, p, ctypes.byref(to), ctypes.byref(o),
                                                          ctypes.byref(h)))
        self.h = h
        n = ctypes.c_int64()
        self.lib.efie_num_unknowns(self.h, ctypes.byref(n))
        self.N = n.value
        self.k = k

    def _stream(self):
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def _vec(self, x):
        import torch
        if x.dtype != torch.complex128 or not x.is_cuda or not x.is_contiguous():
            raise ValueError("expected a contiguous complex128 CUDA tensor")
        if x.shape[-1] != self.N:
            raise ValueError("last dimension must equal the number of unknowns")
        return ctypes.c_void_p(x.data_ptr())

    @staticmethod
    def _rows(x, what):
        """x as [n, N]: a vector [N] becomes one row."""
        if x.dim() not in (1, 2):
            raise ValueError(f"{what} must be [N] or [n, N] (got {list(x.shape)})")
        return x if x.dim() == 2 else x.unsqueeze(0)

    @classmethod
    def _same_rows(cls, x2, y, what):
        """The caller's second array as [n, N], holding exactly the rows of x2.
        The C ABI takes one count for both arrays and no sizes, so this check
        is the only guard against reading or writing past the shorter one."""
        y2 = cls._rows(y, what)
        if tuple(y2.shape) != tuple(x2.shape):
            raise ValueError(f"{what} must have the shape of the input, {list(x2.shape)} (got {list(y.shape)})")
        return y2

    def info(self):
        i = PlanInfo()
        _check(self.lib, self.lib.efie_plan_info(self.h, ctypes.byref(i)), self.h)
        return {f: getattr(i, f) for f, _ in PlanInfo._fields_}

    def rwg_edges(self):
        e = np.zeros((self.N, 2), dtype=np.int32)
        t = np.zeros((self.N, 2), dtype=np.int32)
        _check(self.lib, self.lib.efie_rwg_edges(self.h, e.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                                 t.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))), self.h)
        return e, t

    def rhs_planewave(self, khat, pol):
        import torch
        khat, pol = planewave_args(khat, pol)
        out = torch.empty((khat.shape[0], self.N), dtype=torch.complex128, device="cuda")
        _check(self.lib, self.lib.efie_rhs_planewave(
            self.h, khat.shape[0], khat.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            pol.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.c_void_p(out.data_ptr()),
            self._stream()), self.h)
        return out

    def rhs_planewave_noalloc(self, khat, pol, out):
        """Plane-wave right-hand sides into the caller's complex128 CUDA tensor
        `out` [n, N] without any device allocation by the library."""
        khat, pol = planewave_args(khat, pol, tuple(out.shape), self.N)
        _check(self.lib, self.lib.efie_rhs_planewave_noalloc(
            self.h, khat.shape[0], khat.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            pol.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), self._vec(out), self._stream()), self.h)
        return out

    def matvec(self, x, y=None, fp64=False):
        import torch
        x2 = self._rows(x, "x")
        if y is None:
            y2 = torch.empty_like(x2)
            out = y2 if x.dim() == 2 else y2[0]
        else:
            y2, out = self._same_rows(x2, y, "y"), y
        fn = self.lib.efie_matvec_fp64 if fp64 else self.lib.efie_matvec
        _check(self.lib, fn(self.h, self._vec(x2), self._vec(y2), x2.shape[0], self._stream()), self.h)
        return out

    def matvec_host(self, x, y=None):
        """y = T x with x, y complex128 CPU tensors [n_rhs, N] (pin them for the
        copies to overlap the products).  Ordered on the current CUDA stream;
        synchronize it before reading y."""
        import torch
        x2 = x if x.dim() == 2 else x.unsqueeze(0)
        if x2.device.type != "cpu" or x2.dtype != torch.complex128 or not x2.is_contiguous():
            raise ValueError("x must be a contiguous complex128 CPU tensor")
        if x2.shape[-1] != self.N:
            raise ValueError("last dimension must equal the number of unknowns")
        if y is None:
            y = torch.empty_like(x2, pin_memory=x2.is_pinned())
        y2 = y if y.dim() == 2 else y.unsqueeze(0)
        if y2.shape != x2.shape or y2.dtype != torch.complex128 or not y2.is_contiguous():
            raise ValueError("y must be a contiguous complex128 CPU tensor shaped like x")
        _check(self.lib, self.lib.efie_matvec_host(self.h, ctypes.c_void_p(x2.data_ptr()),
                                                   ctypes.c_void_p(y2.data_ptr()), x2.shape[0],
                                                   self._stream()), self.h)
        return y

    def matvec_parts(self, x):
        import torch
        x2 = self._rows(x, "x")
        yA = torch.empty_like(x2)
        yV = torch.empty_like(x2)
        _check(self.lib, self.lib.efie_matvec_parts(self.h, self._vec(x2), self._vec(yA), self._vec(yV),
                                                    x2.shape[0], self._stream()), self.h)
        return (yA, yV) if x.dim() == 2 else (yA[0], yV[0])

    def solve(self, rhs, tol=1e-6, x=None):
        import torch
        r2 = self._rows(rhs, "rhs")
        if x is None:
            x2 = torch.empty_like(r2)
            sol = x2 if rhs.dim() == 2 else x2[0]
        else:
            x2, sol = self._same_rows(r2, x, "x"), x
        infos = (SolveInfo * r2.shape[0])()
        rc = _check(self.lib, self.lib.efie_solve(self.h, self._vec(r2), self._vec(x2), r2.shape[0], tol, infos,
                                                  self._stream()), self.h)
        out = [{f: getattr(i, f) for f, _ in SolveInfo._fields_} for i in infos]
        return sol, out, rc

    # ---- learned preconditioner (not part of the paper)
    N_PARAMS = 25218

    def precond_harvest(self, rhs, restart=10, n_cycles=4):
        """Residual/error pairs from the plain solver's restarted GMRES iterates."""
        import torch
        r2 = self._rows(rhs, "rhs")
        n = r2.shape[0] * n_cycles
        R = torch.empty((n, self.N), dtype=torch.complex128, device="cuda")
        Ee = torch.empty_like(R)
        _check(self.lib, self.lib.efie_precond_harvest(self.h, self._vec(r2), r2.shape[0], restart, n_cycles,
                                                       ctypes.c_void_p(R.data_ptr()), ctypes.c_void_p(Ee.data_ptr()),
                                                       self._stream()), self.h)
        return R, Ee

    def precond_train(self, r, e, epochs=10, lr=1e-3, seed=0, objective="residual"):
        if r.dim() != 2:
            raise ValueError(f"r must be [n_pairs, N] (got {list(r.shape)})")
        e = self._same_rows(r, e, "e")
        losses = (ctypes.c_double * max(epochs, 0))()
        obj = {"error": 0, "residual": 1}[objective]
        _check(self.lib, self.lib.efie_precond_train(self.h, self._vec(r), self._vec(e), r.shape[0], epochs, lr,
                                                     seed, obj, losses, self._stream()), self.h)
        return list(losses)

    def precond_save(self, path):
        _check(self.lib, self.lib.efie_precond_save(self.h, path.encode()), self.h)

    def precond_load(self, path):
        _check(self.lib, self.lib.efie_precond_load(self.h, path.encode()), self.h)

    def precond_enable(self, on: bool):
        _check(self.lib, self.lib.efie_precond_enable(self.h, 1 if on else 0), self.h)

    def precond_params(self, new=None):
        out = np.zeros(self.N_PARAMS, dtype=np.float32)
        pin = None
        if new is not None:
            new = np.ascontiguousarray(new, dtype=np.float32).ravel()
            if new.size != self.N_PARAMS:
                raise ValueError(f"expected {self.N_PARAMS} parameters (got {new.size})")
            pin = new.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        _check(self.lib, self.lib.efie_precond_params(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                      pin, self.N_PARAMS), self.h)
        return out

    def precond_apply(self, r):
        import torch
        r2 = self._rows(r, "r")
        z = torch.empty_like(r2)
        _check(self.lib, self.lib.efie_precond_apply(self.h, self._vec(r2), self._vec(z), r2.shape[0],
                                                     self._stream()), self.h)
        return z if r.dim() == 2 else z[0]

    def precond_gradient(self, r, e):
        g = np.zeros(self.N_PARAMS, dtype=np.float32)
        loss = ctypes.c_double()
        _check(self.lib, self.lib.efie_precond_gradient(self.h, self._vec(r), self._vec(e),
                                                        g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                        ctypes.byref(loss), self._stream()), self.h)
        return g, loss.value

    def autotune(self, n_rhs):
        """Returns (rhs_chunk, mac_variant, near_variant) chosen for this handle."""
        c, m, n = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(self.lib, self.lib.efie_autotune(self.h, n_rhs, self._stream(), ctypes.byref(c), ctypes.byref(m),
                                                ctypes.byref(n)), self.h)
        return c.value, m.value, n.value

    def autotune_set(self, rhs_chunk: int, mac_variant: int, near_variant: int = 0):
        _check(self.lib, self.lib.efie_autotune_set(self.h, rhs_chunk, mac_variant, near_variant), self.h)

    def transform_schedule(self, schedule=None):
        """Sets the transform schedule (0 line passes, 1 forward y-z passes
        fused, 2 forward and inverse fused, 3 both fused on 9-spline levels
        only) when given; returns the handle's schedule."""
        if schedule is not None:
            _check(self.lib, self.lib.efie_transform_schedule_set(self.h, int(schedule)), self.h)
        v = ctypes.c_int()
        _check(self.lib, self.lib.efie_transform_schedule_get(self.h, ctypes.byref(v)), self.h)
        return v.value

    def profile(self, enable: bool):
        _check(self.lib, self.lib.efie_profile(self.h, 1 if enable else 0), self.h)

    def profile_read(self):
        """{class name: (total ms, launches)} of the recorded kernel classes."""
        out = {}
        i = 0
        while True:
            name = ctypes.create_string_buffer(64)
            ms = ctypes.c_double()
            nl = ctypes.c_int64()
            rc = self.lib.efie_profile_read(self.h, i, name, 64, ctypes.byref(ms), ctypes.byref(nl))
            if rc == EFIE_EINVAL:
                break
            _check(self.lib, rc, self.h)
            out[name.value.decode()] = (ms.value, nl.value)
            i += 1
        return out

    def launch_count(self):
        n = ctypes.c_int64()
        _check(self.lib, self.lib.efie_launch_count(self.h, ctypes.byref(n)), self.h)
        return n.value

    SETUP_PHASES = ("plan", "tables", "near", "far")

    def setup_times(self):
        """Wall seconds of the setup phases: host plan (with exact moments),
        device tables, FP64 near-field assembly, far-field products."""
        t = (ctypes.c_double * 4)()
        n = ctypes.c_int()
        _check(self.lib, self.lib.efie_setup_times(self.h, t, 4, ctypes.byref(n)), self.h)
        return {k: float(t[i]) for i, k in enumerate(self.SETUP_PHASES[:n.value])}

    def close(self):
        if getattr(self, "h", None):
            self.lib.efie_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
