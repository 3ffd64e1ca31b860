"""GB300-native (sm_103a) library for the RIOT incremental 4D-Var inner loop.

The compute path is the CUDA library ``libriot.so`` (sources in ``csrc/``,
C ABI in ``include/riot.h``), built in-tree by ``build.build()``; ``riot``
is its Python binding.
"""
