"""GB300 ICON-type nonhydrostatic dynamical core: Python binding of the C-ABI.

The binding (``_binding.py``) only marshals arguments to libicondycore.so;
``build.py`` compiles that library.  Attribute access on this package
(``paper_2608_21150_gb300.Dycore``, ``.icon_dycore_step``, ...) loads the
binding and raises ImportError if the library has not been built: there is
no fallback implementation.
"""
import importlib


def __getattr__(name):
    if name.startswith("__") or name == "_binding":
        raise AttributeError(name)
    return getattr(importlib.import_module(__name__ + "._binding"), name)
