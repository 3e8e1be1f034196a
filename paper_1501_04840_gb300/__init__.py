"""GB300-native dynamic optimal transport with mixed boundary conditions.

Solver of the discrete Benamou-Brenier problem of Fitschen, Laus & Steidl
(arXiv 1501.04840) by the primal-dual iteration of their Algorithm 1, on RGB
image grids (Neumann x, y; periodic colour) and periodic hue histograms.  All
numerical work runs in the CUDA library ``libdynot.so`` (C ABI in
``include/dynot.h``); :mod:`.binding` only marshals arguments.
"""
from .binding import (BC_NEUMANN, BC_PERIODIC, OT_ECUDA, OT_EINVAL, OT_EMASS, OT_ENOMEM, OT_ENOTCONV,  # noqa: F401
                      OT_ENUMERIC, OT_ETIMEOUT, OT_EUNSUPPORTED, OT_OK, PREC_FP32, PREC_FP64, PREC_MIXED, Batch, Grid,
                      OTError, Plan, Stats, abi_version, grid, hue_grid, load_library, prox, rgb_grid)
