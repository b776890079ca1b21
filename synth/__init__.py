"""Seeded synthetic inputs (meshes, DG operators, aggregate hierarchies,
right-hand sides, candidate matrices) used by both the CUDA path's tests and
benchmark and by the CPU oracle.  It holds none of the multigrid method's
arithmetic."""
