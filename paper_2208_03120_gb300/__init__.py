"""NFFT-accelerated multi-marginal Sinkhorn on GB300 (sm_103a).

The compute path lives in the C-ABI shared library ``libmotfft.so`` built from
``csrc/`` (see ``include/motfft.h``); :mod:`paper_2208_03120_gb300.motfft` is
its thin ctypes binding.  :mod:`paper_2208_03120_gb300.workloads` draws the
seeded synthetic inputs.  Importing the package loads nothing; the library is
loaded on first use of the binding and a missing library is an error.
"""
__all__ = ["motfft", "workloads"]
