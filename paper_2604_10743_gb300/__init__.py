"""GB300-native EM/TM stress, void and IR-drop engine (EMSpice 3 hot path).

The compute path is libems.so (hand-written CUDA for sm_103a) behind the C ABI
in include/ems.h; this package only marshals arguments to it.
"""
from ._abi import (EMS_F64, EMS_F32, EMS_BE, EMS_KRYLOV, EMS_AUTO, EmsError, lib)  # noqa: F401


def Engine(*args, **kwargs):
    from .engine import Engine as _E
    return _E(*args, **kwargs)
