"""B300-native coverage gradient field + LQR step (arXiv 2511.11514).

The compute path is the CUDA C-ABI library ``libcov.so`` (sources under
``csrc/``, declarations in ``include/cov.h``); ``binding`` marshals torch
tensors into its calls.  ``workloads`` draws the seeded synthetic inputs.
The binding is imported lazily so that input generation works on machines
without the built library.
"""
import importlib

__all__ = ["binding", "workloads", "build_lib", "autotune", "autograd"]


def __getattr__(name):
    if name in ("binding", "build_lib", "autotune", "autograd"):
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
