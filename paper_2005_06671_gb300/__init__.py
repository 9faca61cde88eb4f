"""GB300-native soft shadows on curved terrain (arXiv 2005.06671 hot path).

The compute path is the CUDA library ``libsoftshadow.so`` (sm_103a), built
in-tree by ``paper_2005_06671_gb300.build`` and called through its C ABI
(include/softshadow.h).  This package only marshals PyTorch tensors into it.
"""
from .shadow import (Heightfield, Sun, ShadowFn, shadow, ss_build_maxmip, ss_shadow_forward,
                     ss_shadow_uniform, ss_shadow_backward, maxmip_bytes, maxmip_layout,
                     maxmip_views, maxmip_stats, maxmip_nonfinite_count, version, Batch,
                     ss_batch_submit, ss_view_rays, ss_shadow_greedy, ss_shade)

__all__ = ["Heightfield", "Sun", "ShadowFn", "shadow", "ss_build_maxmip", "ss_shadow_forward",
           "ss_shadow_uniform", "ss_shadow_backward", "maxmip_bytes", "maxmip_layout",
           "maxmip_views", "maxmip_stats", "maxmip_nonfinite_count", "version", "Batch",
           "ss_batch_submit",
           "ss_view_rays", "ss_shadow_greedy", "ss_shade"]
