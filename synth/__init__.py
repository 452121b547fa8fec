"""Seeded synthetic inputs shared by the oracle and the CUDA path's tests.

Holds no arithmetic of the GW method itself: it only draws H0(k), S(k),
V^{kk'}(Q), picks the sampled Matsubara integers and names the workloads.
"""
from .generate import (CONFIGS, SEED_BASE, config_seed, matsubara_indices, v_slab,
                       make_config_system, batch_configs, make_batch_system,
                       make_system, kmesh_size, LazyV, device_V)

__all__ = ["CONFIGS", "SEED_BASE", "config_seed", "matsubara_indices", "v_slab", "make_config_system",
           "batch_configs", "make_batch_system",
           "make_system", "kmesh_size", "LazyV", "device_V"]
