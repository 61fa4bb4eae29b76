"""GB300 (sm_103a) EBSD indexing by FFT cross-correlation template matching
with orientation refinement (Foden, Collins, Wilkinson & Britton,
arXiv 1807.11313).

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/ebsdxcf.h``); ``xcf`` is its thin binding.  Importing this package
loads nothing; the first call loads (and if needed builds) the library.
"""
from .xcf import (  # noqa: F401
    Context, Library, XcfError, geometry, xcf_build_library, xcf_build_library_images,
    xcf_correlate_all, xcf_crop, xcf_disorientation, xcf_index, xcf_index_refine, xcf_index_refine_host,
    xcf_options, xcf_geometry, xcf_prep, xcf_project, xcf_refine, load, library_path,
    xcf_profile_enable, xcf_profile_read, STAGES, xcf_index_noalloc, xcf_noalloc_max_patterns,
    xcf_build_library_ex, xcf_screen_topk, xcf_rescore, xcf_refine_best, xcf_index_maps, XCF_LIB_SCREEN,
    XCF_MAPS_GRAPH, Net, xcf_net_num_params, xcf_net_create, xcf_net_forward, xcf_net_loss_grad, xcf_net_adam,
    xcf_propose, xcf_index_learned, xcf_index_precision, xcf_set_scratch_limit, xcf_scratch_bytes,
    XCF_LIB_NDP, XCF_LIB_NO_SPECTRA, xcf_index_ndp, xcf_rotation_scan, XCF_SO3_DEDUP, xcf_so3_grid,
    xcf_nearest_disorientation, xcf_fp32_fma_rate, xcf_maps_get_tuning, xcf_maps_set_tuning, XCF_BODY_REG,
    XCF_BODY_ROUNDS, XCF_BODY_SMEM, XCF_BODY_OCT,
)
