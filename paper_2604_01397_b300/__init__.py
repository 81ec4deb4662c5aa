"""B300-native EXaCTz: bounded-iteration topology correction of decompressed
scalar fields (extremum graph and contour tree preservation), as hand-written
sm_103a CUDA kernels behind a C ABI (include/exactz.h).

The Python layer only marshals torch tensors to that ABI; importing the package
loads the in-tree CUDA library and raises if it has not been built.
"""
from . import _native
from .api import (  # noqa: F401
    MODES,
    STATUS,
    DIRECTIONS,
    EVENTS,
    ExactzError,
    Server,
    Workspace,
    classify,
    correct,
    correct_batch,
    correct_noalloc,
    cp_order,
    decode_edits,
    decode_edits_stream,
    dims_of,
    encode_edits,
    make_opts,
    version,
)

_native.lib()
