"""GB300-native compact full multigrid (CMG) with linear storage.

The compute path is the CUDA library ``libcmg.so`` (C ABI in include/cmg.h);
``paper_2511_19036_gb300.cmg`` is its thin Python binding.  Build with
``paper_2511_19036_gb300._build.build()``.
"""
__all__ = ["cmg"]
