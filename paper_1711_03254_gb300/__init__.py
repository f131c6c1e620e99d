"""GB300-native two-component Shan-Chen D3Q19 lattice Boltzmann library
(Otomo et al., arXiv:1711.03254).

* ``lbm``        ctypes binding of the C ABI in include/lbm.h (CUDA library
                 ``liblbm_gb300.so``; no CPU fallback);
* ``build``      in-tree nvcc build of that library for sm_103a;
* ``workloads``  seeded synthetic geometries and initial fields.
"""
__all__ = ["lbm", "build", "workloads"]
