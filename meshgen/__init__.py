"""Seeded synthetic simplex meshes (input generation only).

This package produces the triangular and tetrahedral grids that both the CPU
oracle and the CUDA path consume.  It contains no part of the grid-metric
method itself (no directed-area vectors, no dual volumes); the only geometric
test it performs is an orientation predicate used to reject jittered grids
with inverted elements, so that every generated grid is a valid simplex mesh.

Workloads (all on the unit square / unit cube, interior nodes jittered):

* ``tri_square``  -- n x n cells, each split along its (i,j)->(i+1,j+1)
  diagonal into 2 triangles (the structure of the paper's triangular test
  grid, Sec. 5).
* ``kuhn_cube``   -- n^3 hexahedral cells, each split into the 6 Kuhn
  tetrahedra sharing the cell diagonal (the structure of the paper's
  tetrahedral test grid, Sec. 5: 256^3 x 6 tets).
* ``batched_set`` -- many Kuhn cubes of uneven size (deforming / adaptation
  sequences, Sec. 5).
"""

from .generate import (  # noqa: F401
    SEED_BASE,
    Mesh,
    tri_square,
    kuhn_cube,
    single_simplex,
    batched_set,
    workload,
    WORKLOADS,
)
