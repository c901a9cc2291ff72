"""GB300-native one-cell inversion (OCI) for SCB x MB time-dependent slab S_N
transport.  The compute path is the CUDA library `liboci` (C ABI declared in
include/oci.h); `paper_2503_00264_gb300.oci` is its thin ctypes binding and
`paper_2503_00264_gb300.workloads` generates seeded synthetic problems.

Importing the package loads nothing; the binding loads `liboci.so` on first use
and raises if it is missing.
"""
__all__ = ["oci", "workloads"]
