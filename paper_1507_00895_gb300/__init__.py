"""GB300-native ladder dual-fermion hot path (opendf, arXiv:1507.00895).

The compute path lives in ``libdf.so`` (CUDA, sm_103a) behind the C ABI
declared in ``include/df.h``; :mod:`paper_1507_00895_gb300.df` is the thin
ctypes binding over it.  :mod:`paper_1507_00895_gb300.inputs` holds the
seeded synthetic input generators (closed-form Hubbard-atom inputs of
Section "Example I", Eqs. atomic_limit1-4) shared by tests and benchmarks.

Importing this package does not load the CUDA library; ``df`` loads it on
first use and raises if it is missing.
"""

__all__ = ["inputs", "df"]
