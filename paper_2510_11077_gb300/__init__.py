"""GB300-native (sm_103a) batched Kalman-filter likelihood of pulsar-timing-array
data: C-ABI library libargus.so (include/argus.h) plus a thin Python binding.

Modules: ``argus`` (binding), ``inputs`` (seeded synthetic arrays),
``build`` (nvcc build of the library).
"""
