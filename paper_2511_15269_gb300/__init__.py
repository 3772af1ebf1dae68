"""GB300-native evaluation of the adaptive point-charge Laplace FMM of
arXiv 2511.15269 (jaxFMM): device-built median-split tree and level-marching
interaction lists, P2M, rotation-based M2M/M2L/L2L, L2P and the P2P near field
as hand-written CUDA kernels for sm_103a behind a C ABI (include/fmm.h).

The CUDA binding lives in :mod:`paper_2511_15269_gb300.fmm`; importing this
package does not load it.
"""
