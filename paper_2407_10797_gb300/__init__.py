"""GB300-native semi-coherent F-statistic for the hierarchical SmBBH search
(arXiv:2407.10797): CUDA kernels for sm_103a behind a C-ABI library, with a
thin ctypes binding."""
