"""GB300-native SU3_Bench link multiply (arXiv 2103.00571): c[i].link[j] = a[i].link[j] x b[j].

The work runs in libsu3 (hand-written CUDA for sm_103a behind the C ABI of include/su3.h); this
package is its thin Python binding plus the autotuner. PyTorch supplies device memory and streams.
"""
from ._binding import (AOS, AOSOA32, BF16, F16, F32, F32PAIR, F64, FULL18, HOST_AUTO, HOST_DIRECT,  # noqa: F401
                       HOST_STAGED, HYBRID, NATIVE, OP_AN, OP_NA, OP_NN, SOA, TWOROW12,
                       BatchItem, Desc, Handle, Su3Error, array_bytes, check_desc, header_functions, lib,
                       library_path, link_bytes)

__all__ = ["Handle", "Desc", "BatchItem", "Su3Error", "lib", "array_bytes", "link_bytes", "check_desc",
           "F64", "F32", "F16", "BF16", "FULL18", "TWOROW12", "AOS", "AOSOA32", "SOA", "NATIVE", "F32PAIR", "HYBRID",
           "OP_NN", "OP_NA", "OP_AN", "HOST_AUTO", "HOST_DIRECT", "HOST_STAGED",
           "FLOP_PER_SITE", "site_update_bytes"]

#: flop per site update by the paper's convention: 4 links x 27 complex MACs x (4 mul + 4 add)
FLOP_PER_SITE = 864


def site_update_bytes(dtype, repr_in=FULL18, repr_out=None):
    """Algorithmic HBM bytes of one site update: the 4 input links read plus the 4 output links
    written (b is read once per launch and ignored, as the paper does)."""
    repr_out = repr_in if repr_out is None else repr_out
    return 4 * (link_bytes(dtype, repr_in) + link_bytes(dtype, repr_out))
