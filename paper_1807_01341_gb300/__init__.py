"""GB300 (sm_103a) implementation of the SWIFT SPH hot path (arXiv 1807.01341).

The compute lives in the C-ABI library ``libsph_gb300.so`` (``include/sph.h``):
cell build, active marking, drift/kicks, density loop with the smoothing-length
iteration, force loop and time bins, in a plain per-bin launch form and a
batched persistent-kernel + CUDA-graph form.  Submodules: ``build`` (nvcc build
of the library), ``_lib`` (ctypes binding), ``sim`` (torch front end: device
memory and streams only).
"""
