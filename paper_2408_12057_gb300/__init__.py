"""GB300-native Optimised Annealed Importance Sampling (arXiv 2408.12057).

The compute path lives in the CUDA library ``liboais.so`` (sources in
``csrc/``, C-ABI declared in ``include/oais.h``); ``oais.py`` is the thin
ctypes binding that marshals arguments and lets PyTorch provide device memory
and streams.  Import the binding explicitly::

    from paper_2408_12057_gb300 import oais
"""
__all__ = ["workloads", "oais"]
