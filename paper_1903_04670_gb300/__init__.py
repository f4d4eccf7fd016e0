"""GB300-native fast spectral collision operator Q^(pq) of the multi-species
DGFS method (Jaiswal, Hu, Brillon & Alexeenko, PASC'19, arXiv 1903.04670).

The compute path is a C-ABI CUDA library (``csrc/``, built for sm_103a);
``binding`` is a thin ctypes layer over it.  ``workloads`` makes seeded inputs.
"""
__all__ = ["binding", "workloads"]
