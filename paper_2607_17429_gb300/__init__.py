"""GB300-native symmetry-adapted FTLM (arXiv 2607.17429): C-ABI library + thin binding.

The compute path lives in libftlm.so (CUDA for sm_103a plus a C++ host group
module); ``ftlm`` is its ctypes binding.  Import ``paper_2607_17429_gb300.ftlm``
after building (``paper_2607_17429_gb300.build.build()``).
"""
