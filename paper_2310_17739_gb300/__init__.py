"""GB300-native state-vector simulator for deep, fused gate streams with
mid-circuit measurement (arXiv 2310.17739's data-parallel hot path).

The compute path is the native library ``libqsim.so`` (hand-written sm_103a
CUDA kernels behind a C ABI, declared in ``include/qsim.h``).  ``qsim`` is the
ctypes binding; ``workload`` builds seeded synthetic inputs.  Importing the
package loads nothing; ``paper_2310_17739_gb300.qsim`` loads the library and
raises if it is missing.
"""
