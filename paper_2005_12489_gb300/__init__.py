"""GB300-native display-driven tile renderer (HiVision, arXiv 2005.12489).

The compute path lives in ``libhivision.so`` (hand-written CUDA for sm_103a
behind a C ABI, declared in ``include/hivision.h``).  ``hv`` is the thin
ctypes binding with the C names; it only marshals arguments.
"""
from . import hv  # noqa: F401
from .hv import (HV_INDEX_LEARNED, HV_INDEX_RTREE, HV_LAYER_LINES, HV_LAYER_POINTS,  # noqa: F401
                 HV_LAYER_POLYGONS, HV_MODE_COVERAGE, HV_MODE_MASK, HV_MODE_RGBA, HVError)
