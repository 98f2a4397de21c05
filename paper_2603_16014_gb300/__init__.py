"""GB300 fast multitask Gaussian processes (arXiv 2603.16014): exact NLL, gradient and posterior.

The compute path is the CUDA library ``libmtgp_gb300.so`` (C ABI in include/mtgp.h); ``mtgp`` is
its Python binding and ``inputs`` the seeded synthetic inputs.  Import ``mtgp`` explicitly: it
needs the built library and torch.
"""
__all__ = ["build", "inputs", "mtgp"]
