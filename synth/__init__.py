"""Seeded synthetic inputs shared by the CPU oracle, the tests and the benchmark.

This package generates meshes, media, source and receiver positions and plane-wave
parameters only.  It holds none of the scheme's arithmetic (no basis functions,
no quadrature, no operators): every input it returns is a plain array that the
oracle and the CUDA library each consume with their own code.
"""
from .meshes import tri_grid, tet_kuhn, add_slivers, unwrap_elements  # noqa: F401
from .media import layered_2d, homogeneous, gaussian_random_field, lame_from_speeds  # noqa: F401
from .workloads import (  # noqa: F401
    Workload, c1_periodic_pwave, c2_layered_slivers, c3_cube_swave,
    c4_multishot, c4_ragged, c5_adjoint, scaled, ragged_union, permuted,
)
