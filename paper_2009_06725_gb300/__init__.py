"""GB300-native spatio-spectral complex Stokes solver (SCVS, arXiv 2009.06725).

The solver is the CUDA library ``libscvs.so`` (C ABI in include/scvs.h);
``paper_2009_06725_gb300.scvs`` is its thin ctypes binding and
``paper_2009_06725_gb300.build`` compiles it for sm_103a.
"""
