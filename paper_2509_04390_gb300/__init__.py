"""GB300-native streaming partitioned convolution with feedback cancellation.

The compute path is the CUDA engine in ``csrc/`` behind the C ABI of
``include/conv.h``; ``upols`` is its thin ctypes binding.  Importing the
package loads nothing; the binding loads the shared library on first use and
raises if it has not been built.
"""

__all__ = ["upols", "signals"]
