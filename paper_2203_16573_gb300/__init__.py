"""GB300-native solver for the surface-source-extension subproblem of
W. W. Symes, "Efficient Computation of Extended Surface Sources"
(arXiv 2203.16573).

``ssx``       -- the Python binding of the C ABI (include/ssx.h); loads
                 libssx.so on first use and raises if it is missing.
``workloads`` -- seeded synthetic inputs (models, wavelets, geometry).
``build``     -- in-tree nvcc build of libssx.so for sm_103a.
"""
__all__ = ["ssx", "workloads", "build"]
