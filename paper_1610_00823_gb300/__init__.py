"""GB300-native adaptive volume-potential box FMM (the box code of Section 3).

Python binding of the C ABI in include/vfmm.h. Every step of the computation
runs in the CUDA library libvfmm.so; this package only marshals arguments and
hands it torch-allocated device memory and the current CUDA stream. There is no
CPU path: if the library is missing, every call raises.
"""
from .api import (FP64, MIXED, M2L_DENSE, M2L_PLANEWAVE, LISTS, Batch, Graph, Ops, SolveGraph, Tree, evaluate_points, leaf_interpolate, ops_create,
                  schedule, set_schedule,
                  source_sample, tree_build, tree_build_leaves, tree_build_many, tree_build_pull, tree_build_uniform, volume_potential,
                  volume_potential_host, workspace, workspace_size, workspace_status)

__all__ = ["FP64", "MIXED", "M2L_DENSE", "M2L_PLANEWAVE", "LISTS", "Batch", "Graph", "Ops", "SolveGraph", "Tree", "evaluate_points", "leaf_interpolate", "ops_create",
           "schedule", "set_schedule",
           "source_sample",
           "tree_build", "tree_build_leaves", "tree_build_many", "tree_build_pull", "tree_build_uniform", "volume_potential", "volume_potential_host", "workspace",
           "workspace_size", "workspace_status"]
