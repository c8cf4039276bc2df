"""GB300 (sm_103a) hot path of RNN-wave-function variational Monte Carlo.

The kernels live in ``libnqs.so`` (C ABI in ``include/nqs.h``), built in-tree by
``paper_2507_18700_gb300.build``; ``paper_2507_18700_gb300.nqs`` is the Python
binding.  Importing the package does not load the library; calling any binding
function without a built library raises.
"""
