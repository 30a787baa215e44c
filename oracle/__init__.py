"""FP64 CPU oracle of FEWHA's per-frame hot path.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline / reference arm of ``bench.py`` may import anything from this package.
The product path (the CUDA library and its Python binding) never does.
"""

from .fewha_oracle import *  # noqa: F401,F403
