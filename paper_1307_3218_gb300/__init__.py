"""GB300-native multiple Arnoldi (mArnoldi) solver.

The hot path of the mArnoldi method (Hoshi, Yamazaki, Akiyama, arXiv:1307.3218,
Section 2) runs in libmarnoldi, hand-written CUDA for sm_103a behind the C ABI
declared in ``include/marnoldi.h``.  This package holds the CUDA sources
(``csrc/``), their build (``build.py``) and the ctypes binding
(``marnoldi.py``), whose functions carry the C names (``Server`` wraps the
request server, ``marnoldi_server_*``), and the host logic that splits the
columns over ranks with one shared Fermi level (``shard.py``).
"""

from .marnoldi import (MARNOLDI_FP64, MARNOLDI_MIXED, Context, MarnoldiError, Server, load,
                       marnoldi_check_status, marnoldi_column_stats, marnoldi_device_bytes, marnoldi_footprint, marnoldi_gs_shape,
                       marnoldi_set_autotune, marnoldi_count_noalloc, marnoldi_density, marnoldi_density_device,
                       marnoldi_destroy, marnoldi_eigenstate, marnoldi_energy, marnoldi_fermi_at, marnoldi_forces,
                       marnoldi_green,
                       marnoldi_kernel_kinds, marnoldi_level_range, marnoldi_member_energy, marnoldi_set_member_temperatures, marnoldi_set_members,
                       union_of,
                       marnoldi_kernel_stats, marnoldi_last_error, marnoldi_set_allocator,
                       marnoldi_set_batch, marnoldi_set_profiling, marnoldi_setup,
                       marnoldi_set_krylov_graph, marnoldi_krylov_graph_launches,
                       marnoldi_solve, marnoldi_solved_shape, setup_system, use_torch_allocator)

__all__ = [
    "MARNOLDI_FP64", "MARNOLDI_MIXED", "Context", "MarnoldiError", "Server", "load",
    "marnoldi_check_status", "marnoldi_column_stats", "marnoldi_device_bytes", "marnoldi_footprint", "marnoldi_gs_shape",
    "marnoldi_set_autotune", "marnoldi_count_noalloc", "marnoldi_density", "marnoldi_density_device", "marnoldi_destroy",
    "marnoldi_eigenstate", "marnoldi_energy", "marnoldi_fermi_at", "marnoldi_forces", "marnoldi_green", "marnoldi_kernel_kinds",
    "marnoldi_kernel_stats", "marnoldi_level_range", "marnoldi_member_energy", "marnoldi_set_member_temperatures",
    "marnoldi_set_members",
    "union_of",
    "marnoldi_last_error", "marnoldi_set_allocator", "marnoldi_set_batch",
    "marnoldi_set_profiling", "marnoldi_set_krylov_graph", "marnoldi_krylov_graph_launches",
    "marnoldi_setup", "marnoldi_solve", "marnoldi_solved_shape",
    "setup_system", "use_torch_allocator",
]
