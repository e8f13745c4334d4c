"""GB300-native batched critical-node-detection fitness and GA step (GAPA, arXiv 2412.20980).

The compute path is libgapa.so (hand-written sm_103a CUDA kernels behind a C
ABI, declared in include/gapa.h); ``gapa`` is its ctypes binding.
"""
from .gapa import (
    Batch,
    Config,
    Context,
    GapaError,
    Surrogate,
    SurrogateConfig,
    make_surrogate_config,
    run_surrogate,
    EXPORTS,
    FLAG_MU_PLUS_LAMBDA,
    FLAG_ROULETTE,
    FLAG_ROWWISE,
    load,
    make_config,
    preset_config,
    PRESETS,
    threshold,
)

__all__ = ["Batch", "Config", "Context", "GapaError", "Surrogate", "SurrogateConfig", "make_surrogate_config",
           "run_surrogate", "EXPORTS", "FLAG_MU_PLUS_LAMBDA", "FLAG_ROULETTE", "FLAG_ROWWISE", "load", "make_config", "preset_config", "PRESETS", "threshold"]
