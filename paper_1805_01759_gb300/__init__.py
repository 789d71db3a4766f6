"""GB300-native batched complex basis pursuit denoising (RBPG, arXiv 1805.01759).

The compute path is libbpdn.so (CUDA for sm_103a, C ABI in include/bpdn.h);
``paper_1805_01759_gb300.api`` is its thin Python binding.  ``synth`` simulates
seeded input stacks.  Importing this package loads nothing; the binding loads the
library on first use and raises if it has not been built.
"""

__all__ = ["api", "synth", "build"]
