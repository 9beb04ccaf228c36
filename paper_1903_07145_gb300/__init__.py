"""GB300-native inverse path tracing (Azinovic et al., CVPR 2019).

Submodules:
  scenes  -- seeded synthetic scenes (inputs only; no light transport)
  build   -- compiles libipt.so for sm_103a
  _lib    -- ctypes binding of the C ABI in include/ipt.h
  tracer  -- torch-facing wrapper and torch.autograd.Function
"""
import importlib

__all__ = ["scenes", "build", "tracer"]


def __getattr__(name):
    if name in ("scenes", "build", "tracer", "_lib"):
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
