"""GB300-native semi-analytical isogeometric thermal solver (hot path).

The compute path is libsa.so (hand-written CUDA for sm_103a) behind the C
ABI declared in ``include/sa.h``.  This package only marshals arguments
(``_binding``); there is no CPU fallback: importing the binding without the
built library raises ImportError.
"""
from ._binding import *  # noqa: F401,F403
