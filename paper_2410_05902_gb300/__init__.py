"""GB300-native mini-batch kernel k-means (truncated centers, beta learning rate).

The compute path is the CUDA library ``libkkm.so`` (sm_103a), which exports a
plain C ABI declared in ``include/kkm.h``. ``paper_2410_05902_gb300.kkm`` is a
thin ctypes binding over it. ``paper_2410_05902_gb300.inputs`` holds the seeded
synthetic workloads.
"""
__all__ = ["inputs"]
