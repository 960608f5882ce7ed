"""GB300 (sm_103a) THC second-order self-energy library.

The compute path is the C-ABI library ``lib/libthcsigma.so`` (CUDA kernels);
``paper_2404_17744_gb300.thc`` is its thin ctypes binding.  Build with
``python -m paper_2404_17744_gb300.build``.
"""
