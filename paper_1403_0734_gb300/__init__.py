"""GB300-native k-clique counting (FFF_k) and colour-sampling estimation
(cFFF_k): the CUDA library libkc behind the C ABI in include/kc.h, and this
thin Python binding with the same names."""
from .kc import (KC_ALGO_DFS, KC_ALGO_PIVOT, KC_DEVICE_PTRS, KC_PARAM_ALGO, KC_MAX_K, KC_PARAM_LAUNCH_COUNT, KC_PARAM_SMEM_MAX_WORDS,
                 KC_PARAM_WORK_COUNT, KC_VALIDATE, Graph, KcError,
                 build_csr, count, count_batch, count_csr, count_part, count_static, count_device, estimate, estimate_csr, estimate_pairs, export, footprint, get_param,
                 orient, set_param, version)

__all__ = ["KC_ALGO_DFS", "KC_ALGO_PIVOT", "KC_PARAM_ALGO", "Graph", "KcError", "build_csr", "count", "count_batch", "count_part", "count_static", "count_csr", "count_device", "estimate", "estimate_pairs",
           "estimate_csr", "export", "footprint", "orient", "version", "set_param", "get_param", "KC_PARAM_SMEM_MAX_WORDS", "KC_PARAM_LAUNCH_COUNT", "KC_PARAM_WORK_COUNT", "KC_DEVICE_PTRS", "KC_VALIDATE", "KC_MAX_K"]
