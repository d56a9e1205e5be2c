"""CPU oracle for the stabilized multilevel B-spline fast EFIE method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run
anything in this package.  The CUDA library never imports, links or calls it,
and this package never imports the library: the two share no code.  The only
common module is ``efie_inputs`` (seeded mesh and vector generators, no method
arithmetic).

Contents (all FP64 unless a function says otherwise):

* ``geometry``   - RWG functions without edge-length normalization and the star
                   matrix (Sec. II, Sec. VI-A).
* ``quadrature`` - Gauss rules generated at run time (Golub-Welsch), collapsed
                   triangle rules, analytic static potential integrals over flat
                   triangles, and a polar-coordinate brute-force integrator used
                   only to pin the former.
* ``dense``      - dense Galerkin EFIE, T = jk A + (jk)^-1 Sigma V Sigma^T
                   (Eq. discretizedEFIE, Eq. matTA, Eq. matTPhi, Sec. VI-A),
                   plane-wave right-hand side.
* ``mie``        - Mie series surface current of a PEC sphere.
* ``bspline``    - open equidistant knot vectors (Eq. eqknots), Cox-de Boor
                   evaluation, Boehm knot insertion (Sec. IV-B), transfer
                   matrices C, knot-removal stabilization S, B_stab, P (Sec. V-B,
                   Table I).
* ``tree``       - uniform octree, per-level spline counts and buffers
                   (Sec. III-B, IV-C, IV-D), interaction lists.
* ``moments``    - exact RWG and pulse moments by knot-plane clipping (Eq.
                   TAfactor, Sec. VI-A).
* ``fastmv``     - the straightforward multilevel B-spline fast matvec (Eq.
                   TAfactorBspline, Eq. interleveltransfer, Sec. V-B).
* ``nonuniform`` - the same fast matvec on a nonuniform octree (Sec. VII tree
                   rule, Sec. IV-C/D buffer rule for leaves on the parent
                   level, level-consistent near blocks).
* ``factorizations`` - the direct (RWG + divergence moments) and dyadic
                   (3 x 3 Hessian translations) factorizations (Sec. VI), on
                   the uniform and on the nonuniform octree.
* ``krylov``     - plain GMRES / FGMRES.
* ``mpnn``       - FP64 NumPy forward/backward of the learned preconditioner
                   network (not part of the paper).

Functions whose result has no independent pin say "parity unpinned" in their
docstring.
"""
