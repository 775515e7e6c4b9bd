"""FP64 CPU oracle of the eRTIS energyscape chain.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` use it.  It shares no code with the CUDA library.
"""
from .rtis64 import *  # noqa: F401,F403
