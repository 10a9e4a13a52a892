"""GB300-native all-at-once Crank-Nicolson solver with the generalized block alpha-circulant
preconditioner (arXiv 2401.16113).

Submodules: `build` compiles the CUDA library, `aao` binds its C ABI, `workloads` holds the
seeded synthetic problem parameters. Importing the package does not load the library.
"""
