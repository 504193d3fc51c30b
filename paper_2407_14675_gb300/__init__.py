"""GB300 semi-Lagrangian Bellman solver for planar low-thrust orbit transfer.

The solver lives in libdp.so (CUDA, sm_103a) behind the C ABI of
include/dp.h; ``paper_2407_14675_gb300.dp`` is its Python binding and
``paper_2407_14675_gb300.workloads`` holds the seeded synthetic problems.
"""
__all__ = ["dp", "workloads", "build"]
