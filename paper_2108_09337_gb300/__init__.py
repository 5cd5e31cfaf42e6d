"""GB300-native dense LU (tournament pivoting) and Cholesky, after COnfLUX /
COnfCHOX (Kwasniewski et al., SC'21, arXiv 2108.09337).

The compute path is the C-ABI library ``libcf.so`` (CUDA, sm_103a) declared in
``include/cf.h``; :mod:`paper_2108_09337_gb300.cf` is its thin ctypes binding.
Importing this package does not load the library; the first call into
:mod:`.cf` does, and raises if the library is missing.
"""
import importlib

__all__ = ["cf", "inputs"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
