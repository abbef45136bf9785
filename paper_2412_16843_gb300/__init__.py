"""GB300-native CDI + GNBC contact-line solver (arXiv 2412.16843).

The compute path is the CUDA library libcdi.so (C ABI declared in
include/cdi.h); `paper_2412_16843_gb300.cdi` is its thin Python binding.
`paper_2412_16843_gb300.inputs` holds the seeded synthetic inputs.
"""
__all__ = ["cdi", "inputs"]
