"""GB300-native plane-wave H|psi> and block Davidson (libqegb).

The binding lives in ``binding`` and is loaded on first attribute access, so
that ``paper_2104_10502_gb300.build`` can run before the library exists.
Every name of the binding (Context, gsphere, QEError, QE_* constants) is
available from the package.
"""
import importlib


def __getattr__(name):
    if name.startswith("__"):
        raise AttributeError(name)
    return getattr(importlib.import_module(__name__ + ".binding"), name)
