"""GB300 (sm_103a) implementation of the 3DPIFCM hot path.

3DPIFCM segments noisy volumes with fuzzy C-means whose distance carries two
neighbourhood-attraction terms weighted by (lambda, xi), tuning (lambda, xi)
with a particle swarm (Agranonik, Herman, Last, arXiv 2002.01981, Eqs 1-10,
Algorithms 1-2).  The path runs in hand-written CUDA kernels behind the C ABI
of ``include/pifcm.h`` (``libpifcm.so``); ``paper_2002_01981_gb300.ifcm`` is
its Python binding, ``distributed`` splits one swarm across the ranks of a
torch.distributed group, and ``phantoms`` generates the seeded synthetic
inputs.

Submodules are imported on demand so that the input generator and the build
step work on machines without a GPU.
"""
__all__ = ["build", "distributed", "ifcm", "native", "phantoms"]
