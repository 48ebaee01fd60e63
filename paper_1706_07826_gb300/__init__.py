"""GB300 (sm_103a) library for sample-persistence variable reduction (SPVAR,
Alg. 1) and Multi-start SPVAR (Alg. 2) with a simulated-annealing sampler.

The compute path is the C-ABI CUDA library ``libspvar.so`` (``include/spvar.h``);
``spvar`` is its thin Python binding and ``instances`` draws synthetic
problems shaped like the paper's workloads.  Importing this package loads
nothing; the library is loaded on first use and must have been built.
"""
__all__ = ["spvar", "instances"]
