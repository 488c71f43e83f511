"""GB300-native boundary oracle and random walks for spectrahedra
(arXiv 2010.03817).  The compute path is the CUDA library ``libspectra_gb``
behind the C ABI in ``include/spectra_gb.h``; :mod:`.spectra` is its Python
binding and :mod:`.workloads` the seeded synthetic inputs."""

__all__ = ["spectra", "workloads"]
