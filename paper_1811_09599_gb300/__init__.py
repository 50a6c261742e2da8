"""qflex_gb300: single-GPU (GB300, sm_103a) contraction of random-quantum-circuit
tensor networks into output amplitudes (after arXiv:1811.09599, "qFlex").

The compute path is the CUDA library built from csrc/ (C ABI in
include/qflex.h); this package only marshals arguments.  Importing it does not
need a GPU; calling into the library on a machine without one raises.
"""
from ._lib import QFlexError, load  # noqa: F401


def __getattr__(name):
    # lazy import so that `import paper_1811_09599_gb300` stays torch-free
    if name in ("Plan", "QFlexAmplitudes", "permute", "cgemm", "norm", "device_status"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
