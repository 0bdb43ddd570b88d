"""GB300-native Welsch-norm MM non-rigid registration with Anderson
acceleration (Yao et al., arXiv 2206.03410).

The registration runs in hand-written CUDA kernels for sm_103a behind the
C ABI declared in include/nrr.h (library ``_build/libnrr.so``); the submodule
``nrr`` is the ctypes binding with the same function names. Importing this
package does not load the library; the first call does, and raises if it
cannot.
"""
