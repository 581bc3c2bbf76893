"""GB300 damage-diffusion field engine: CUDA C-ABI library (libdd.so) + thin binding.

The computation lives in csrc/ (CUDA for sm_103a) behind include/dd.h; the Python
side only marshals arguments (binding.py) and builds the library (build.py).
"""
__all__ = ["binding", "build", "workloads"]
