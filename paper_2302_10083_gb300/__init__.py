"""GB300-native dense ternary prime-implicant sweep (DenseQMC, arXiv 2302.10083).

The compute path is the CUDA library ``libdqmc.so`` (C ABI in ``include/dqmc.h``);
:mod:`paper_2302_10083_gb300.dqmc` is its thin ctypes binding.  Importing this
package does not load the library; the binding loads it on first use and raises
if it is missing (there is no CPU fallback).
"""
__all__ = ["dqmc", "synth"]
