"""GB300-native arbitrary-shape-surface Fresnel diffraction (Shimobaba, Masuda, Ito).

The computation lives in the CUDA library libasfd.so (C ABI: include/asfd.h);
`capi` binds it with ctypes under the same names, `fresnel.FresnelPlan` is a
small handle over a plan, and `workloads` generates the seeded synthetic inputs.
Importing this package loads nothing; the library is loaded on first use.
"""

__all__ = ["capi", "fresnel", "workloads"]
