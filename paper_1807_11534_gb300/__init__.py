"""GB300 (sm_103a) implementation of the restricted-domain dual formulation of
two-phase TV segmentation (arXiv 1807.11534).

* ``paper_1807_11534_gb300.seg``   -- binding of the C ABI in include/seg.h
  (libseg.so, hand-written CUDA kernels); imported on first use.
* ``paper_1807_11534_gb300.synth`` -- seeded synthetic inputs.
* ``paper_1807_11534_gb300.build`` -- builds libseg.so in-tree for sm_103a.
"""

__all__ = ["seg", "synth", "build"]


def __getattr__(name):
    if name in ("seg", "synth", "build"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
