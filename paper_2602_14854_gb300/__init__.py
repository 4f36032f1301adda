"""GB300-native domain-decomposition dynamical low-rank (DD-DLRA) time step for
the radiative transfer equation (arXiv 2602.14854).

The method runs in the CUDA library ``lib/libddlra.so`` (built from ``csrc/``
by ``build.build()``), called through the C ABI of ``include/ddlra.h``;
``binding`` is its ctypes binding and ``inputs`` builds seeded synthetic
problem data.  Importing the package loads nothing.
"""
__all__ = ["binding", "build", "inputs"]
