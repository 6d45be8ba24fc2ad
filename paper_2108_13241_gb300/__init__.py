"""D2Q9 BGK stream-and-collide on one GB300 (sm_103a): dense and tiled-sparse
grids, two-lattice and in-place AA patterns, FP64 / FP32 / FP16-shifted
storage, and a hand-written adjoint.

The compute path is the CUDA library ``csrc/`` builds (``liblbm.so``); the
Python modules only marshal arguments to its C ABI.

  lbm       -- ctypes binding with the C names (lbm_create, lbm_step, ...) and
               the ``LBM`` convenience class;
  autograd  -- ``LBMFunction`` (torch.autograd.Function) with sqrt(T)
               checkpointing on top of lbm_backward;
  inputs    -- seeded synthetic geometries and initial fields;
  build     -- compiles the CUDA library for sm_103a.

Submodules are imported on demand so that importing ``inputs`` alone does not
load the CUDA library.
"""
