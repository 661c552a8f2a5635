"""GB300 (sm_103a) DMTS-NC: dual-level RESPA molecular dynamics with a
conservative message-passing potential at the outer step and a distilled
non-conservative direct-force model at the inner steps.

The compute path is the CUDA library libdmts.so (C ABI in include/dmts.h);
`core` is its torch-facing binding and `synth` generates seeded inputs.
Importing the package does not load the library; the first call does, and
raises if it cannot.
"""


def build():
    from . import buildlib
    return buildlib.build()


def __getattr__(name):
    if name in ("core", "synth", "_lib"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
