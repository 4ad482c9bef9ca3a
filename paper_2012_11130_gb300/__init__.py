"""GB300 (sm_103a) per-patch SRHD fluid update of arXiv 2012.11130.

The compute path is libsrhd.so (CUDA C ABI, include/srhd.h); this package is
its thin Python binding plus seeded synthetic workloads. Importing the
package does not load the library; ``srhd`` does, and raises if it is
missing.
"""
from . import build  # noqa: F401

__all__ = ["build", "srhd", "workloads"]
