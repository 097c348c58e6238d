"""GB300-native wall-modelled lattice Boltzmann LES hot path.

`paper_2506_21804_gb300.lbm` binds the CUDA C-ABI library (liblbm.so); importing this package
does not load it, so the seeded input generators in `paper_2506_21804_gb300.inputs` stay usable
on machines without a GPU.
"""
