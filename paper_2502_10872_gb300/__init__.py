"""GB300-native corotational hinge-based thin plates/shells (arXiv 2502.10872): Python binding of the C ABI.

The compute path is the CUDA library ``libshells.so`` (sm_103a) built from ``csrc/`` by
:func:`paper_2502_10872_gb300._build.build`; this package only marshals arguments (see
:mod:`paper_2502_10872_gb300.binding`). The six bending models are named as in the paper: EP, ES (edge-based
hinge), FP, FS (FVM hinge), SP, SS (smoothed hinge); P = plate (rest-flat), S = shell (rest-curved).
"""
from .binding import *  # noqa: F401,F403
from .binding import (Batch, Handle, LibraryNotBuilt, ShellError, create_from_scenario, load_library,  # noqa: F401
                      make_options)


def build(verbose: bool = False) -> str:
    """Compile ``libshells.so`` in-tree for sm_103a and return its path."""
    from ._build import build as _b
    return _b(verbose=verbose)
