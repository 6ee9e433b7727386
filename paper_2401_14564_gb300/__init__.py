"""GB300 (sm_103a) Probe-Particle Model hot path: FF grid assembly, relaxed FIRE
scan with trilinear interpolation, and Giessibl df conversion, as CUDA kernels
behind the C ABI of include/pp.h.

Submodules load lazily so that the generators (`synth`) import without a GPU:
  pp     ctypes binding of libpp.so (same entry-point names as pp.h)
  afm    Simulator / afm(): device buffers + the three stages, host end-to-end
  synth  seeded synthetic workloads (inputs only)
  build  nvcc build of libpp.so
"""
import importlib

__all__ = ["pp", "afm", "synth", "build"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
