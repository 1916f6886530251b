"""GB300-native Voronoi cells of every particle (the per-particle hot path of PARAVT, arXiv:1601.06429).

The compute path is the CUDA library ``libvt_gb300.so`` behind the C ABI in
``include/vt_gb300.h``; :mod:`.binding` exposes the same entry points to
Python, :mod:`.autograd` the differentiable volume, :mod:`.inputs` the seeded
synthetic point sets, and :mod:`.build` compiles the library for sm_103a.
"""
from . import inputs  # noqa: F401  (no CUDA needed)


def build(force: bool = False) -> str:
    from .build import build as _b

    return _b(force=force)
