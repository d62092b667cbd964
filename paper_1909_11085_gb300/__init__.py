"""GB300-native Stokes layer-potential sums (single layer, double layer,
their superposition, the FMM near field over U-lists, batched suspensions,
the adjoint) and the steps around them (check-point quadrature, the
boundary-integral operator, the near-zone search, the octree and the FMM's
far field) behind the C ABI of include/stokesgpu.h.

The compute path is libstokesgpu.so (hand-written CUDA for sm_103a); this
package only marshals PyTorch tensors into it.  Build the library with
paper_1909_11085_gb300.build.build().
"""
from .ops import (sl, dl, sldl, p2p, batched, sldl_grad, StokesLayerFn,  # noqa: F401
                  DirectPlan, P2PPlan, BatchedPlan, CheckpointPlan, BIEPlan, upsample_patches,
                  near_patch_search, octree, fmm_tree_arrays, fmm_tree_args, fmm_operators,
                  fmm_m2l_spectra, FmmFarPlan, FmmPlan)

__all__ = ["sl", "dl", "sldl", "p2p", "batched", "sldl_grad", "StokesLayerFn", "DirectPlan",
           "P2PPlan",
           "BatchedPlan", "CheckpointPlan", "BIEPlan", "upsample_patches",
           "near_patch_search", "octree", "fmm_tree_arrays", "fmm_tree_args", "fmm_operators",
           "fmm_m2l_spectra", "FmmFarPlan", "FmmPlan"]
