"""GB300-native pipe-flow Navier-Stokes time step (Openpipeflow method).

The CUDA library `libopf.so` (built from csrc/) carries the whole time step;
`paper_1705_03838_gb300.opf` is its thin ctypes binding.  `inputs` holds the
seeded synthetic-state recipe.
"""
