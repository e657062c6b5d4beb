"""GB300-native hot path of the compressed key sort (Kwon et al., arXiv 2009.11543).

``ck``        thin ctypes binding of libck (include/ck.h), same names as the C ABI
``pipeline``  index reconstruction (extract -> sort -> bulk load) over the binding
``metrics``   the paper's compression / sort key ratios and the roofline byte counts
``build``     nvcc build of libck.so for sm_103a
"""
__all__ = ["ck", "pipeline", "metrics", "build"]
