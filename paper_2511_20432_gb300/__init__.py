"""GB300-native semi-analytical isogeometric thermal solver (hot path).

The compute path is libsa.so (hand-written CUDA for sm_103a) behind the C
ABI declared in ``include/sa.h``.  This package only marshals arguments
(``_binding``); there is no CPU fallback: touching any API name without the
built library raises ImportError.  ``paper_2511_20432_gb300.build`` compiles
the library and does not need it.
"""
import importlib


def __getattr__(name):
    if name.startswith("__") or name in ("build", "_binding"):
        raise AttributeError(name)
    return getattr(importlib.import_module(__name__ + "._binding"), name)
