"""FP64 CPU oracle for the Elfpie gradient step (arXiv 2209.14671).

This package is TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The CUDA library never imports, links or calls it, and it shares no code with the
CUDA path; the only module both sides read is the seeded input generator
``paper_2209_14671_gb300.inputs``, which holds no arithmetic of the method.
"""
from .elfpie_oracle import *  # noqa: F401,F403
