"""GB300 all-mode sparse MTTKRP engine (Wijeratne, Kannan, Prasanna, CF '24).

The computation lives in a CUDA shared library with a C ABI
(``include/spmttkrp.h``); this package only builds it (``_build``) and binds
it (``binding``).  There is no CPU fallback.
"""
from .binding import Plan, SpmError, check_elements, declared_functions, lib  # noqa: F401

__all__ = ["Plan", "SpmError", "check_elements", "declared_functions", "lib"]
