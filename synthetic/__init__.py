"""Seeded synthetic inputs shared by the oracle tests and the GPU path.

This package draws operators, panels and random vectors; it contains none of
the sparse-product arithmetic that the oracle or the CUDA library implement.
"""
from ._native import build  # noqa: F401
from .structures import (AtomSystem, BlockPattern, block_diagonal, morton_order,  # noqa: F401
                         neighbor_pattern, periodic_images, random_pattern, zincblende_cell)
from .workloads import (Workload, amorphous, batched_uneven, decay_scale, domain, nnz_row_scale,  # noqa: F401
                        normal_panel, rademacher_panel, random_values, stream_key,
                        symmetric_values, tiny_multispecies, zincblende,
                        PeriodicWorkload, image_values, zincblende_crystal)
