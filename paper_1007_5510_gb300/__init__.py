"""GB300-native randomized block-Lanczos PCA (Halko, Martinsson, Shkolnisky,
Tygert): CUDA library behind a C-ABI (include/rpca.h) and a thin binding."""
from .rpca import (PCA, RpcaError, pca, fused_pass, t_pass, qr_inplace, small_svd, gaussian,
                   kernel_launches, load_library, F64, F32, BF16, FP8E4M3)

__all__ = ["PCA", "RpcaError", "pca", "fused_pass", "t_pass", "qr_inplace", "small_svd",
           "gaussian", "kernel_launches", "load_library", "F64", "F32", "BF16", "FP8E4M3"]
