"""B300-native global pose alignment (BundleFusion, Dai et al., Sec. 4.2-4.4).

The solver runs in the CUDA library ``libbf.so`` behind the C ABI of
``include/bf.h``; this package is its thin Python binding.  Importing it does not
touch the GPU; creating a :class:`Context` does.
"""
from ._lib import (Context, BFError, default_params, verify_params, lib, LIB_PATH, EXPORTS, tc_probe,  # noqa: F401
                   BF_PTR_HOST, BF_PTR_DEVICE, BF_STORE_FP32, BF_STORE_BF16, BF_STORE_FP16,
                   BF_PRECOND_BLOCK_JACOBI, BF_PRECOND_JACOBI, BF_PREC_MIXED, BF_PREC_FP32,
                   BF_FLAG_SINGULAR_BLOCK, BF_FLAG_EMPTY_FRAME, BF_FLAG_PCG_BREAKDOWN,
                   BF_PCG_AUTO, BF_PCG_CTA, BF_PCG_GRID, BF_PCG_CLUSTER, BF_SPARSE_BLOCKS, BF_SPARSE_MATFREE,
                   BF_TILE_AUTOTUNE)
