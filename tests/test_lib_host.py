"""CPU tests of the library: the C ABI loads and exports every declared symbol,
and its host-side planning (octree, per-level spline counts, interaction and
near lists, projector and transfer matrices) agrees with the oracle."""
import os
import re

import numpy as np
import pytest

import efie_inputs as E

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build_library_only()
    import paper_2606_13482_gb300 as G
    return G, G.load_library()


def test_exports_every_declared_symbol(lib):
    G, L = lib
    hdr = open(os.path.join(ROOT, "include", "efie.h")).read()
    declared = set(re.findall(r"^(?:int|const char \*)\s*(efie_\w+)\s*\(", hdr, re.M))
    assert declared == set(G.EXPORTED_SYMBOLS)
    for name in declared:
        assert hasattr(L, name), name


def test_plan_matches_oracle(lib):
    G, _ = lib
    from oracle import fastmv
    from oracle.geometry import build_rwg
    from oracle.tree import build_tree, interaction_lists
    for (freq, r, k, p, delta, levels) in [(8, 0.5, 2 * np.pi, 3, 0.1, 2), (10, 0.5, 2 * np.pi * 1.7, 2, 0.08, 3),
                                           (8, 0.5, 2 * np.pi, 5, 0.1, 1), (14, 0.5, 2 * np.pi * 2.5, 3, 0.06, 2),
                                           (14, 0.5, 2 * np.pi * 0.5, 3, 0.06, 3)]:
        V, T = E.icosphere(freq, r)
        info, lv = G.plan(V, T, k, p, delta, levels)
        m = build_rwg(V, T)
        tr = build_tree(m, k, p, delta, levels)
        assert info["depth"] == tr.D and info["top_level"] == tr.top
        assert np.allclose(info["root_lo"], tr.root_lo, atol=0, rtol=0)
        for L in lv:
            O = tr.levels[L["level"]]
            assert (L["s"], L["sb"], L["sp"], L["shat"]) == (O.s, O.sb, O.sp, O.shat)
            assert L["n_boxes"] == len(O.boxes)
            assert L["n_far_pairs"] == len(interaction_lists(tr, L["level"])[0])
            assert L["nfft"] >= 2 * L["shat"] - 1
        op = fastmv.BsplineEFIE.__new__(fastmv.BsplineEFIE)
        op.tree = tr
        nb, rb, tb = fastmv.BsplineEFIE.near_masks(op)
        assert info["near_nnz_A"] == int(nb[rb[:, None], rb[None, :]].sum())
        assert info["near_nnz_V"] == int(nb[tb[:, None], tb[None, :]].sum())


def test_plan_matrices_match_oracle(lib):
    """P = B_stab^-1 S and the knot-insertion transfers C^L, C^R, built by the
    library's host code, against the oracle's construction (both the
    increasing-s and the constant-s rule)."""
    G, _ = lib
    from oracle.bspline import S_REMOVE, open_knots, projector, restriction_matrix
    from oracle.geometry import build_rwg
    from oracle.tree import build_tree
    for (freq, r, k, p, delta, levels) in [(14, 0.5, 2 * np.pi * 2.5, 3, 0.06, 2),
                                           (14, 0.5, 2 * np.pi * 0.5, 3, 0.06, 3),
                                           (14, 0.5, 2 * np.pi * 0.5, 5, 0.06, 2)]:
        V, T = E.icosphere(freq, r)
        tr = build_tree(build_rwg(V, T), k, p, delta, levels)
        for ell in range(tr.D, tr.top - 1, -1):
            L = tr.levels[ell]
            Pref = projector(open_knots(0.0, float(L.sp - p), L.sp, p), p, S_REMOVE[p])[0]
            Pm = G.plan_matrix(V, T, k, p, delta, levels, ell, 0)
            assert np.abs(Pm - Pref).max() < 1e-12 * max(1, np.abs(Pref).max())
            if ell > tr.top:
                pa = tr.levels[ell - 1]
                rr = int(round(pa.delta / L.delta))
                Up = open_knots(-pa.sb * rr, (pa.s - p + pa.sb) * rr, pa.sp, p)
                CL = restriction_matrix(Up, open_knots(-L.sb, (L.s - p) + L.sb, L.sp, p), p)
                CR = restriction_matrix(Up, open_knots((L.s - p) - L.sb, 2 * (L.s - p) + L.sb, L.sp, p), p)
                assert np.abs(G.plan_matrix(V, T, k, p, delta, levels, ell, 1) - CL).max() < 1e-14
                assert np.abs(G.plan_matrix(V, T, k, p, delta, levels, ell, 2) - CR).max() < 1e-14


def test_plan_moments_match_oracle(lib):
    """Exact leaf-spline moments built by the library's host planner
    (each triangle clipped and integrated once per leaf box, its tiles shared
    by its RWGs and its pulse) against the oracle's per-function clipping and
    collapsed Gauss rule, for p = 2, 3, 5; and the divergence moments of the
    direct factorization."""
    G, _ = lib
    from oracle.geometry import build_rwg
    from oracle.moments import pulse_moments, rwg_moments
    from oracle.tree import build_tree
    rng = np.random.default_rng(11)
    for (freq, r, k, p, delta, levels) in [(8, 0.5, 2 * np.pi, 3, 0.1, 2), (10, 0.5, 2 * np.pi * 1.7, 2, 0.08, 3),
                                           (8, 0.5, 2 * np.pi, 5, 0.1, 1)]:
        V, T = E.icosphere(freq, r)
        m = build_rwg(V, T)
        keys = m.edges[:, 0].astype(np.int64) * len(V) + m.edges[:, 1]
        assert np.all(np.diff(keys) > 0)  # canonical order: edges sorted by (lo, hi)
        tr = build_tree(m, k, p, delta, levels)
        ids = rng.choice(m.N, 48, replace=False).astype(np.int32)
        ref = rwg_moments(m, tr, ids)
        got = G.plan_moments(V, T, k, p, delta, levels, 0, ids)
        assert got.shape == ref.shape
        assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()
        tids = rng.choice(m.Nt, 48, replace=False).astype(np.int32)
        ref = pulse_moments(m, tr, tids)
        got = G.plan_moments(V, T, k, p, delta, levels, 1, tids)
        assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()
    # divergence moments of the direct factorization, in the RWG's box
    from oracle.factorizations import divergence_moments
    ref = divergence_moments(m, tr, ids)
    got = G.plan_moments(V, T, k, p, delta, levels, 2, ids)
    assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()
    with pytest.raises(G.EfieError):
        G.plan_moments(V, T, k, p, delta, levels, 3, ids)
    with pytest.raises(G.EfieError):
        G.plan_moments(V, T, k, p, delta, levels, 1, np.array([m.Nt], np.int32))


def test_plan_adaptive_matches_oracle(lib):
    """Nonuniform octree planned by the library's host code against the
    oracle's (`oracle.nonuniform`): per-level boxes, leaves, spline counts,
    translated pairs, leaf functions, and the near RWG / triangle pairs.  The
    library reports them from the plan its device pipeline runs
    (efie_setup_adaptive): interaction lists, leaves in Morton order, and the
    near blocks over the leaves."""
    G, _ = lib
    from oracle import nonuniform as NU
    from oracle.geometry import build_rwg
    from oracle.tree import interaction_lists
    two = E.merge_meshes(E.icosphere(8, 0.3, center=(-1.0, 0, 0)), E.icosphere(5, 0.8, center=(1.0, 0.1, 0.05)))
    for (freq, r, k, me, top) in [(14, 0.5, 2 * np.pi, 60, 2), (14, 0.5, 2 * np.pi * 2.5, 60, 2),
                                  (12, 0.5, 2 * np.pi, 40, 2), (None, None, 2 * np.pi, 30, 2)]:
        # the last case: a fine small sphere beside a coarse large one, leaves on levels 2, 3 and 4
        V, T = E.icosphere(freq, r) if freq else two
        m = build_rwg(V, T)
        tr = NU.build_adaptive_tree(m, k, 3, max_elems=me, top=top)
        lv, nr, nt = G.plan_adaptive(V, T, k, 3, max_elems=me, top=top)
        assert [L["level"] for L in lv] == list(range(tr.top, tr.D + 1))
        for L in lv:
            O = tr.levels[L["level"]]
            assert (L["s"], L["sb"], L["sp"], L["shat"]) == (O.s, O.sb, O.sp, O.shat)
            assert L["n_boxes"] == len(O.boxes) and L["n_leaves"] == int(tr.is_leaf[L["level"]].sum())
            assert L["n_far_pairs"] == len(interaction_lists(tr, L["level"])[0])
            assert L["n_leaf_rwg"] == int((tr.rwg_level == L["level"]).sum())
            assert L["n_leaf_tri"] == int((tr.tri_level == L["level"]).sum())
            assert L["h"] == pytest.approx(O.h, rel=1e-15) and L["delta"] == pytest.approx(O.delta, rel=1e-15)
        nb = NU.near_leaf_pairs(tr)
        _, _, rl, tl = NU.leaf_index(tr)
        assert nr == int(nb[rl[:, None], rl[None, :]].sum())
        assert nt == int(nb[tl[:, None], tl[None, :]].sum())
    with pytest.raises(G.EfieError):
        G.plan_adaptive(*E.icosphere(14, 0.5), 2 * np.pi, 3, max_elems=60, top=4)


def test_plan_adaptive_near_and_moments_match_oracle(lib):
    """Leaves, near-leaf lists and per-leaf exact moments of the nonuniform
    tree, built by the library's host code, against `oracle.nonuniform`
    (moments of every function in its own leaf's splines, sampled ids)."""
    G, _ = lib
    from oracle import nonuniform as NU
    from oracle.geometry import build_rwg
    from oracle.moments import pulse_moments, rwg_moments
    V, T = E.icosphere(14, 0.5)
    m = build_rwg(V, T)
    k = 2 * np.pi
    tr = NU.build_adaptive_tree(m, k, 3, max_elems=60, top=2)
    lvl, ijk, ptr, src = G.plan_adaptive_near(V, T, k, 3, max_elems=60, top=2)
    olvl, oijk, _, _ = NU.leaf_index(tr)
    assert np.array_equal(lvl, olvl) and np.array_equal(ijk, oijk)
    nb = np.zeros((len(lvl), len(lvl)), dtype=bool)
    for x in range(len(lvl)):
        nb[x, src[ptr[x]:ptr[x + 1]]] = True
        assert np.all(np.diff(src[ptr[x]:ptr[x + 1]]) > 0)
    assert np.array_equal(nb, NU.near_leaf_pairs(tr))
    rng = np.random.default_rng(4)
    # the moments efie_setup_adaptive uploads: the sphere above (leaves on two
    # levels), and a fine small sphere beside a coarse large one (three levels)
    two = E.merge_meshes(E.icosphere(8, 0.3, center=(-1.0, 0, 0)), E.icosphere(5, 0.8, center=(1.0, 0.1, 0.05)))
    for (Vc, Tc, me, n_lv) in ((V, T, 60, 2), (two[0], two[1], 30, 3)):
        mc = m if Vc is V else build_rwg(Vc, Tc)
        trc = tr if Vc is V else NU.build_adaptive_tree(mc, k, 3, max_elems=me, top=2)
        for kind, n in ((0, mc.N), (1, mc.Nt)):
            flv = trc.rwg_level if kind == 0 else trc.tri_level
            # up to 20 sampled functions from every level that holds leaves
            ids = np.concatenate([rng.choice(np.nonzero(flv == ell)[0], min(20, int((flv == ell).sum())),
                                             replace=False) for ell in np.unique(flv)]).astype(np.int32)
            blocks, levels = G.plan_adaptive_moments(Vc, Tc, k, 3, kind, ids, max_elems=me, top=2)
            assert np.array_equal(levels, flv[ids]) and len(set(levels)) == n_lv
            for ell in set(levels.tolist()):
                sel = np.nonzero(levels == ell)[0]
                view = NU._LevelView(trc, ell)
                ref = (rwg_moments if kind == 0 else pulse_moments)(mc, view, ids[sel])
                got = np.stack([blocks[i] for i in sel])
                assert got.shape == ref.shape
                assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()


def test_invalid_inputs(lib):
    G, _ = lib
    V, T = E.icosphere(4, 0.5)
    with pytest.raises(G.EfieError) as e:
        G.plan(V, T[:-1], 2 * np.pi, 3, 0.1, 1)          # open mesh
    assert e.value.code == -1
    with pytest.raises(G.EfieError):
        G.plan(V, T, 2 * np.pi, 7, 0.1, 1)               # p out of range
    with pytest.raises(G.EfieError):
        G.plan(V, T, 2 * np.pi, 3, 0.1, 9)               # levels beyond depth + 1
    with pytest.raises(G.EfieError):
        G.plan(V, T, 2 * np.pi, 3, 0.03, 1)              # buffers close the far gap
    Tbad = T.copy()
    Tbad[0] = Tbad[0][[0, 2, 1]]
    with pytest.raises(G.EfieError):
        G.plan(V, Tbad, 2 * np.pi, 3, 0.1, 1)            # inconsistent orientation
    with pytest.raises(G.EfieError):
        G.plan_adaptive(V, T[:-1], 2 * np.pi, 3)          # open mesh
    with pytest.raises(G.EfieError):
        G.plan_adaptive(V, T, 2 * np.pi, 3, max_elems=-1, max_prot=np.inf, top=1, max_depth=5)  # buffers
    # entry points that take a handle reject a NULL one without touching a device
    import ctypes
    _, L = lib
    x = (ctypes.c_double * 4)()
    assert L.efie_matvec_host(None, x, x, 1, None) == G.EFIE_EINVAL
    assert L.efie_setup_times(None, x, 4, None) == G.EFIE_EINVAL
    assert L.efie_launch_count(None, None) == G.EFIE_EINVAL
    assert L.efie_transform_schedule_set(None, 0) == G.EFIE_EINVAL
    sched = ctypes.c_int(-1)
    assert L.efie_transform_schedule_get(None, ctypes.byref(sched)) == G.EFIE_EINVAL and sched.value == -1


def test_setup_without_gpu_fails_loudly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    G, _ = lib
    V, T = E.icosphere(4, 0.5)
    with pytest.raises(G.EfieError) as e:
        G.EFIE(V, T, 2 * np.pi, 3, 0.1, 1)
    assert e.value.code == -3
    with pytest.raises(G.EfieError) as e:
        G.EFIE(V, T, 2 * np.pi, 3, 0.1, 1, factorization=G.EFIE_FACT_DIRECT)
    assert e.value.code == -3
    for fact in (G.EFIE_FACT_DYADIC,):
        with pytest.raises(G.EfieError) as e:
            G.EFIE(V, T, 2 * np.pi, 3, 0.1, 1, factorization=fact)
        assert e.value.code == -3
    with pytest.raises(G.EfieError) as e:
        G.EFIE(V, T, 2 * np.pi, 3, tree=dict(max_elems=30, top=2))
    assert e.value.code == -3


def test_factorization_option_checked_first(lib):
    # an unknown factorization is rejected before any device work (EINVAL,
    # with or without a GPU); the option sits at the end of efie_options
    import ctypes
    G, _ = lib
    V, T = E.icosphere(4, 0.5)
    with pytest.raises(G.EfieError) as e:
        G.EFIE(V, T, 2 * np.pi, 3, 0.1, 1, factorization=7)
    assert e.value.code == -1 and "factorization" in str(e.value)
    assert G.Options.factorization.offset == ctypes.sizeof(G.Options) - 8
    # the nonuniform tree takes the star factorization only; bad tree options
    # are rejected as well, both before any device work
    tree = dict(max_elems=30, top=2)
    for fact in (G.EFIE_FACT_DIRECT, G.EFIE_FACT_DYADIC):
        with pytest.raises(G.EfieError) as e:
            G.EFIE(V, T, 2 * np.pi, 3, tree=tree, factorization=fact)
        assert e.value.code == -1 and "star" in str(e.value)
    with pytest.raises(G.EfieError) as e:
        G.EFIE(V, T, 2 * np.pi, 3, tree=dict(max_prot=-1.0))
    assert e.value.code == -1
    with pytest.raises(ValueError):
        G.EFIE(V, T, 2 * np.pi, 3)
    with pytest.raises(ValueError):
        G.EFIE(V, T, 2 * np.pi, 3, tree=dict(max_elem=30))


def test_planewave_argument_checks(lib):
    """The C ABI takes no sizes for the plane-wave arrays, so the binding
    checks them: khat and pol must both be [n, 3], and an output given by the
    caller must be [n, N]; mismatches are rejected before any library call."""
    G, _ = lib
    kh, pol = G.planewave_args([0, 0, -1.0], [1.0, 0, 0])
    assert kh.shape == (1, 3) and pol.shape == (1, 3) and kh.dtype == np.float64
    kh, pol = G.planewave_args(np.zeros((4, 3)), np.ones((4, 3)), (4, 100), 100)
    assert kh.flags.c_contiguous and pol.shape == (4, 3)
    for bad in [(np.zeros((4, 3)), np.zeros((3, 3)), None, None),      # short pol
                (np.zeros((4, 2)), np.zeros((4, 2)), None, None),      # not 3-vectors
                (np.zeros((4, 3)), np.zeros((4, 3)), (3, 100), 100),   # short output
                (np.zeros((4, 3)), np.zeros((4, 3)), (100,), 100),     # 1-D output
                (np.zeros((4, 3)), np.zeros((4, 3)), (4, 99), 100)]:   # wrong N
        with pytest.raises(ValueError):
            G.planewave_args(*bad)


def test_plan_adaptive_near_pointer_capacity(lib):
    """near_ptr holds n_leaves + 1 entries; a capacity of n_leaves is rejected."""
    G, L = lib
    import ctypes
    V, T = E.icosphere(14, 0.5)
    m, keep = G._mesh(V, T)
    o = G.TreeOptions(60, 0.25, 2, 0, 0)
    nl, nz = ctypes.c_int64(), ctypes.c_int64()
    assert L.efie_plan_adaptive_near(ctypes.byref(m), 2 * np.pi, 3, ctypes.byref(o), ctypes.byref(nl),
                                     ctypes.byref(nz), None, None, 0, None, None, 0) == 0
    ptr = np.zeros(nl.value + 1, np.int64)
    ip = ptr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    assert L.efie_plan_adaptive_near(ctypes.byref(m), 2 * np.pi, 3, ctypes.byref(o), None, None, None, None,
                                     nl.value, ip, None, 0) == G.EFIE_EINVAL
    assert L.efie_plan_adaptive_near(ctypes.byref(m), 2 * np.pi, 3, ctypes.byref(o), None, None, None, None,
                                     nl.value + 1, ip, None, 0) == 0
    assert ptr[-1] == nz.value


class _DeviceArray:
    """Stands in for a contiguous complex128 CUDA tensor of a given shape
    (shape checks only: nothing reads its memory)."""

    def __init__(self, *shape):
        import torch
        self.shape = tuple(shape)
        self.dtype = torch.complex128
        self.is_cuda = True

    def dim(self):
        return len(self.shape)

    def is_contiguous(self):
        return True

    def unsqueeze(self, d):
        assert d == 0
        return _DeviceArray(1, *self.shape)

    def data_ptr(self):
        return 0


class _NoCalls:
    """A library whose every entry point fails the test: the binding must
    reject the arguments before it calls one."""

    def __getattr__(self, name):
        raise AssertionError(f"{name} was called with arguments the binding should reject")


def test_vector_argument_checks(lib):
    """The C ABI's products, solves and training calls take one count for an
    input and an output array and no sizes, so the binding checks that a
    caller-given output (or second input) holds exactly the input's rows and
    that every array is [N] or [n, N]; a parameter vector must hold the
    network's parameter count.  Mismatches are ValueErrors before any
    library call."""
    G, _ = lib
    N = 100
    h = G.EFIE.__new__(G.EFIE)
    h.lib, h.h, h.N = _NoCalls(), None, N
    D = _DeviceArray
    bad_products = [(D(4, N), D(3, N)),      # short output
                    (D(4, N), D(N)),         # one row for four
                    (D(N), D(2, N)),         # two rows for one
                    (D(4, N), D(4, N - 1)),  # wrong N
                    (D(2, 2, N), D(2, 2, N))]  # not [n, N]
    for x, y in bad_products:
        with pytest.raises(ValueError):
            h.matvec(x, y)
        with pytest.raises(ValueError):
            h.solve(x, 1e-6, y)
    with pytest.raises(ValueError):
        h.precond_train(D(8, N), D(7, N))
    with pytest.raises(ValueError):
        h.precond_train(D(N), D(N))
    with pytest.raises(ValueError):
        h.precond_params(np.zeros(h.N_PARAMS - 1, np.float32))
    with pytest.raises(ValueError):
        h.matvec_parts(D(1, 1, N))
    # matching shapes get through to the library
    for x, y in [(D(4, N), D(4, N)), (D(N), D(N)), (D(N), D(1, N))]:
        with pytest.raises(AssertionError):
            h.matvec(x, y)
        with pytest.raises(AssertionError):
            h.solve(x, 1e-6, y)
    with pytest.raises(AssertionError):
        h.precond_train(D(8, N), D(8, N))
    with pytest.raises(AssertionError):
        h.precond_params(np.zeros(h.N_PARAMS, np.float32))
    # a batch: one input and one output per member, of the member's shape
    h2 = G.EFIE.__new__(G.EFIE)
    h2.lib, h2.h, h2.N = _NoCalls(), None, 2 * N
    b = G.Batch.__new__(G.Batch)
    b.lib, b.handles, b.b = _NoCalls(), [h, h2], None
    for xs, ys in [([D(2, N)], [D(2, N)]),                                  # one member missing
                   ([D(2, N), D(3, 2 * N)], [D(2, N), D(2, 2 * N)]),        # short output
                   ([D(2, N), D(3, N)], [D(2, N), D(3, N)]),                # wrong N for member 1
                   ([D(N), D(3, 2 * N)], [D(N), D(3, 2 * N)])]:             # not [n, N]
        with pytest.raises(ValueError):
            b.matvec(xs, ys)
    with pytest.raises(AssertionError):
        b.matvec([D(2, N), D(3, 2 * N)], [D(2, N), D(3, 2 * N)])
