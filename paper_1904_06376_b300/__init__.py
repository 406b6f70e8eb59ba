"""bfx: FP32-accurate GEMM, LU and iterative-refinement solves from bfloat16
pieces on B300 tensor cores (Henry, Tang & Heinecke, ARITH 2019).

This package is a thin binding over the C-ABI library ``libbfx.so`` (built
in-tree from ``csrc/`` by ``build.py``; declarations in ``include/bfx.h``).
Every computation runs in the library's sm_103a kernels; the Python layer only
marshals torch tensors (device memory, streams) into pointers and sizes.
There is no CPU fallback: without the built library every call raises.
"""
from ._bfx import (  # noqa: F401
    BFX_FP32,
    BFX_X1,
    BFX_X3,
    BFX_X5,
    BFX_X6,
    BFX_X8,
    BFX_X9,
    Batch,
    BatchConfig,
    batch_autotune,
    BfxError,
    GEMM_PIECES,
    GMRES_MAX_M,
    IrParams,
    device_error,
    dot_bf16xN,
    gemm_bf16xN,
    gemm_bf16xN_f64,
    gemm_bf16xN_fused,
    gemm_presplit,
    gemm_workspace_size,
    lib,
    LOWP_BF16,
    LOWP_FP16,
    LOWP_FP32,
    lowp_lu_ir_batched,
    lu_bf16xN,
    solve_ir,
    solve_ir_async,
    measure_fma_peak,
    decode_ir_result,
    solve_ir_workspace_size,
    library_path,
    num_sms,
    Server,
    sgemm_simt,
    split,
    split_transpose,
    split_pair,
    version,
)
