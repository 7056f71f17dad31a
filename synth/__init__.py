"""Seeded synthetic inputs shared by the CPU oracle and the CUDA search path."""
from .meshes import (MeshGrid, MeshPair, Planted, build_pair, config1, config1_independent,
                     config2, config3, independent_pair,
                     config4_pair, config4_sizes, config5, config_seed, family_pair,
                     tri_vertex_ij, SEED_BASE, SurfacePair, layered_pair, layered_s_grid)

__all__ = ["MeshGrid", "MeshPair", "Planted", "build_pair", "config1", "config1_independent",
           "config2", "config3", "independent_pair",
           "config4_pair", "config4_sizes", "config5", "config_seed", "family_pair",
           "tri_vertex_ij", "SEED_BASE", "SurfacePair", "layered_pair", "layered_s_grid"]
