"""CPU oracle for the batched Kalman-filter likelihood (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path.

* ``kalman``: plain FP64 C implementation of the O(N) Kalman recursion and a
  complex-step gradient (``kalman.c``), loaded through ctypes.
* ``dense``: the plain definition the recursion reaches exactly, the dense
  multivariate-normal log-density of the residual vector (numpy, Cholesky).
* ``exact``: the dense definition in exact rational arithmetic for tiny cases.
* ``mlp``: FP32 forward/backward of the surrogate network on BF16 operands.
"""
