"""GB300 (sm_103a) pass-through brain connectivity: the hot path of FastCod
(Bian et al., "FastCod: Fast Brain Connectivity in Diffusion Imaging",
arXiv 2302.09247, Section 2, Algorithms 1-2).

    paper_2302_09247_gb300.build    -- compiles csrc/*.cu into _lib/libfastcod.so
    paper_2302_09247_gb300.fastcod  -- ctypes binding of include/fastcod.h

The computation runs only in the CUDA library; importing ``fastcod`` fails
when the library is missing.
"""
