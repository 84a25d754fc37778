"""Block r1-sparse Jacobian hot path on GB300 (sm_103a).

The CUDA library (``libsts.so``, C ABI declared in ``include/sts.h``) is loaded
lazily by :mod:`paper_2403_09198_gb300.binding`; importing this package does not
touch the GPU.  :mod:`paper_2403_09198_gb300.inputs` builds seeded synthetic
workloads and holds none of the method's arithmetic.
"""
__all__ = ["inputs"]
