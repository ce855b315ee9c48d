"""GB300 (sm_103a) engine for exact tensor-network contraction along a fixed path.

The compute path lives in the CUDA library libtn_gb300.so (C ABI: include/tn.h);
this package is its thin Python binding. See `binding` for the wrappers.
"""
from .binding import (Plan, Server, Batch, TnError, check, last_error, make_policy, lib, LIB_PATH,
                      TN_OK, TN_ERR_INVALID, TN_ERR_UNSUPPORTED, TN_ERR_OOM, TN_ERR_CUDA,
                      TN_ERR_BUSY, TN_ERR_TIMEOUT, TN_ERR_NOT_READY,
                      TN_C64_FP32_SIMT, TN_C64_TF32, TN_C64_3XTF32, TN_C64_BF16X3,
                      TN_R32_FP32_SIMT, TN_R32_TF32, TN_R32_3XTF32, TN_R32_BF16X3,
                      TN_CLASS_SIMT, TN_CLASS_STREAM, TN_CLASS_TC, TN_CLASS_SPLITK, TN_CLASS_PERM,
                      CLASS_NAMES)

__all__ = ["Plan", "Server", "TnError", "check", "last_error", "make_policy", "lib", "LIB_PATH"]
