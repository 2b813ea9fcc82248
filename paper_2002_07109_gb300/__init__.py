"""GB300-native BOUNCE velocity-jump molecular dynamics (arXiv 2002.07109).

The compute path is the C-ABI CUDA library ``libbounce.so`` (declared in
``include/bounce.h``); ``paper_2002_07109_gb300.bounce`` is its thin ctypes
binding.  ``paper_2002_07109_gb300.water`` builds seeded synthetic inputs.
Importing this package does not load the CUDA library; importing
``paper_2002_07109_gb300.bounce`` does, and fails loudly if it is missing.
"""
__all__ = ["water", "bounce"]
