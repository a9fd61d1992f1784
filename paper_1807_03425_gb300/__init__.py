"""GB300 (sm_103a) implementation of the Secant-Avoidance Projection (SAP)
hot path (Kvinge, Farnell, Kirby, Peterson, arXiv:1807.03425).

The compute lives in ``libsap.so`` (hand-written CUDA kernels behind the C ABI
of ``include/sap.h``).  This package is the thin Python binding: ``capi``
mirrors the C entry points one-to-one (same names, argument marshalling only)
and ``Sap`` wraps a handle.  There is no CPU fallback: if the shared library
is missing or no GPU is present, calls raise.
"""
from .capi import (SapError, Sap, SapBatch, ShardSap, load_library, library_path,  # noqa: F401
                   PLAIN, RESTRUCTURED, UPDATE_LITERAL, UPDATE_ANGLE,
                   SPLIT_FP16, SPLIT_BF16, F32, BF16, F64, KERNEL_CLASSES)
