"""FP64 CPU oracle for octree TV-L1 range-data fusion (Kehl et al., BMVC 2016).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run
anything in this package.  The product path (the CUDA library and its binding)
never calls it, and this package imports nothing from the product path: the two
share no code.  The only shared module is the seeded input generator
(``paper_1608_07411_gb300.scenes``), which the tests call, not this package.

Plain, slow, obviously correct NumPy/SciPy in float64.  Each function cites the
passage of the paper it restates; where the paper is silent the reading taken
is stated in the docstring.

Modules
  morton     Morton keys of the linear octree (bit interleaving)
  tsdf       Eq. 1 truncated signed distances and the binary weights
  octree     Eq. 2 top-down construction, face neighbours, split/join
  operators  level-aware forward-difference gradient, divergence, step sizes
  solver     normalised TV-L1 energy (Eq. 5), its primal-dual solver, gap
  dense      an independent dense-grid solver (the fully refined special case)
  mlp        the per-leaf warm-start network (features, forward, gradient, Adam)
  descent    the paper's own solver: gradient descent on the eps-L1 energy
             (Eq. 4-6, Sec. 4 schedule)
  quantisation  Eq. 7 quantisation error between a dense and an octree field
  mesh       zero level set of the fused field as a triangle mesh (Sec. 3.3)
  frames     per-frame TSDF octrees as the data-term source (Fig. 4, Table 1)

Parity unpinned: nothing in the oracle reproduces the paper's printed results
(Tables 1-2, the accuracy figures), which need the paper's datasets and its
gradient-descent solver.
"""
