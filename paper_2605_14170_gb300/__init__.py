"""GB300-native Multiple-Bases BP List Decoder (MBBP-LD).

``mbbp``   ctypes binding of the C ABI in ``include/mbbp.h`` (the CUDA library
           ``libmbbp.so``, built by ``build.build()``).
``inputs`` seeded workloads: BB and GB check matrices, random errors, LLRs.
``learn``  WMS training and learned-vs-plain comparison (launch sequencing).
``shard``  shot ranges per rank and the counter / timing reductions.

The binding is imported lazily so that ``inputs`` can be used without the
compiled library.
"""
__all__ = ["mbbp", "inputs", "build", "learn", "shard"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
