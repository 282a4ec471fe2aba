"""GB300 (sm_103a) MSPCG solver for the even-odd Moebius domain-wall-fermion system.

After J. Tu, "Solving DWF Dirac Equation Using Multisplitting Preconditioned
Conjugate Gradient" (LATTICE2018, arXiv:1811.08488).

* ``paper_1811_08488_gb300.dwf``       ctypes binding of the C ABI (include/dwf.h)
* ``paper_1811_08488_gb300.build``     nvcc build of libdwf.so (in-tree)
* ``paper_1811_08488_gb300.synthetic`` seeded SU(3) gauge fields and sources

The binding loads libdwf.so on first use and raises if it has not been built;
there is no CPU fallback.
"""
