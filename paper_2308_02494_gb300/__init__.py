"""GB300-native (sm_103a) APMGSRN point query: forward, backward, density loss,
Adam, batched domain-decomposition bricks and a headless ray-marching renderer.

The compute runs in ``libsrn.so`` (hand-written CUDA kernels behind a C ABI,
declared in ``include/srn.h``).  ``paper_2308_02494_gb300.srn`` is the thin
ctypes binding; importing this package does not load the library, so the
seeded input generators in ``synth`` work on machines without a GPU.
"""
__all__ = ["synth", "srn"]
