"""GB300 library for the server-side hot path (Mask -> Comp) of the HE-based
private database query of arXiv 2408.17063, with client-side Decomp.

The compute path is the CUDA library ``_lib/libpdq.so`` (C ABI in
``include/pdq.h``); ``pdq`` is its thin ctypes binding.  Import the binding
explicitly (``from paper_2408_17063_gb300 import pdq``); it raises if the
library was not built (``paper_2408_17063_gb300.build.build()``).
"""
