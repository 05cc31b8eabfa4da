"""GB300 tensor-train solver for the k-eigenvalue neutron transport problem
(arXiv 2309.03347): a thin ctypes binding over libkeig_tt.so (include/keig.h).

Every computation runs in the library's CUDA kernels; this package only
marshals arguments.  PyTorch supplies the device, the CUDA stream and device
tensors for bulk data.  There is no CPU fallback: if the library or a CUDA
device is missing, the calls raise.
"""
from ._lib import (  # noqa: F401
    TT_OK, TT_EINVAL, TT_ENOMEM, TT_ECUDA, TT_ENOCONV, TT_ETIMEOUT, TT_ENONFINITE,
    TT_OP_H, TT_OP_S, TT_OP_F, TT_MV_EXACT, TT_MV_AMEN, TT_FP64, TT_FP32_REFINED, TT_TF32_SPLIT, TT_BF16_SPLIT,
    KeigError, Context, TorchCachingAllocator, TTVec, TTOp, lib_path, load,
    tt_ctx_create, tt_vec_create, tt_op_create, tt_round, tt_matvec, tt_solve_local, tt_solve_dmrg,
    tt_build_operator, keig_fixed_point, keig_default_opts, tt_scalar_flux, tt_dot_noalloc,
    keig_sensitivities, keig_k_function, keig_j_function, keig_batch, keig_alpha, keig_gpt, keig_slab_fixed_point,
    tt_measure_fma_peak, tt_gemm_f32,
)
