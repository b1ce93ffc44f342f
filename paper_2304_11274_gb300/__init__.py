"""GB300-native TPFA residual/Jacobian assembly (arXiv 2304.11274, Section 3).

The compute path is the CUDA library ``libtpfa.so`` (C ABI in include/tpfa.h),
built in-tree for sm_103a by ``paper_2304_11274_gb300.build``.  Importing the
package does not load the library; the first ``Grid`` does, and fails loudly
if it has not been built.
"""
__version__ = "1.0.0"


def __getattr__(name):
    if name in ("Grid", "Mesh", "Ensemble", "TPFAError"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
