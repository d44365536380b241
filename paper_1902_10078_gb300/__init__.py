"""GB300-native banded SPD operators and their adjoints (arXiv 1902.10078).

The compute path is the CUDA library ``csrc/`` built into ``_libbanded.so``
behind the C ABI declared in ``include/banded.h``.  ``binding`` marshals
arguments to it, ``autograd`` wraps the operators as
``torch.autograd.Function``s, and ``workloads`` synthesises seeded inputs.
Importing the package loads nothing; the library is loaded on first use and
raises if it has not been built.
"""
__all__ = ["binding", "autograd", "workloads", "batch", "losses"]
