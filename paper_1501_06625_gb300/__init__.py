"""GB300-native hot path of polynomial homotopy continuation in complex
double-double and quad-double arithmetic (after Verschelde & Yu, 2015).

Submodules, imported on first use:
  libph  -- Python binding of the C ABI in include/ph.h (libph.so, sm_103a)
  build  -- compiles libph.so in tree
  synth  -- seeded synthetic workloads
  monodromy -- monodromy loops through the serving loop (the degree of a
               solution set, Section 4.2)
"""
import importlib

__all__ = ["libph", "build", "synth", "monodromy"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
