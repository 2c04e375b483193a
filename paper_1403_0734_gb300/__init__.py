"""GB300-native k-clique counting (FFF_k), colour-sampling (cFFF_k) and
pair-sampling estimation: the CUDA library libkc behind the C ABI in
include/kc.h, and this thin Python binding with the same names."""
from . import kc as _kc
from .kc import (CLASS_NAMES, Batch, Graph, KcError, TuningCache, build_csr, count, count_batch, count_csr, count_device,
                 count_part, count_part_device, count_static, estimate, estimate_csr, estimate_pairs, export, footprint, get_param,
                 list_cliques, list_runs, orient, round2_bytes, set_param, set_tuning, tune, version)

_consts = {name: getattr(_kc, name) for name in dir(_kc) if name.startswith("KC_")}
globals().update(_consts)

__all__ = ["CLASS_NAMES", "Batch", "Graph", "KcError", "TuningCache", "build_csr", "count", "count_batch", "count_csr",
           "count_device", "count_part", "count_part_device", "count_static", "estimate", "estimate_csr", "estimate_pairs", "export",
           "footprint", "get_param", "list_cliques", "list_runs", "orient", "round2_bytes", "set_param", "set_tuning", "tune",
           "version", *sorted(_consts)]
