"""B300 (sm_103a) sparse-coefficient Gaussian splatting: the rendering and query path of
LangSplatV2 (arXiv 2507.07136) behind a C ABI (``include/lsv2.h``).

Modules:
  build     nvcc build of ``_build/liblsv2.so`` (all kernels, sm_103a)
  _lib      ctypes binding with the ABI's function names
  pipeline  torch buffers + call sequence (project, bin_sort, splat, decode, query)
"""
from .build import LIB, build  # noqa: F401
