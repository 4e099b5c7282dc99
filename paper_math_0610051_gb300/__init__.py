"""GB300 (sm_103a) library for applying discrete Fourier integral operators.

The method is the wedge-factorised algorithm of Candes, Demanet and Ying,
"Fast Computation of Fourier Integral Operators": polar wedges (Sec. 1.3), a
randomized low-rank separation of the residual phase (Sec. 3.2), and a
type-2 nonuniform FFT per wedge and rank term (Sec. 3.4); the adjoint uses
the type-1 transform (Sec. 3.5).

The compute path lives in the CUDA shared library ``libfio.so`` (C ABI in
``include/fio.h``).  ``fio`` is its Python binding; importing this package
does not load the library (``synth`` is usable without a GPU).
"""

__all__ = ["fio", "synth"]
