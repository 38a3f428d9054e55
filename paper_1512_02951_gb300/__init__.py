"""GB300-native selective protection of RGB bitmaps (DCT 8x8 -> int16 -> zigzag split ->
AES-128-CTR on the confidential fragment), after Sect. 6.3.1 of "Data Protection: Combining
Fragmentation, Encryption, and Dispersion".

The compute path is the CUDA library libfds.so (C ABI in include/fds.h); `api` is its thin
torch binding.  Importing this package does not load the library; the first call does, and
fails loudly if it has not been built.
"""
from . import synth  # noqa: F401  (seeded inputs; no method arithmetic)


def __getattr__(name):
    if name in ("api", "_lib", "build"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
