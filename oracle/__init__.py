"""FP64 CPU oracle for the moment-based Gaussian rasterizer (MB3DGS).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_2512_11800_gb300``) never imports it and
shares no code with it; the only common module is the seeded input
generator ``scenes``.
"""
from .mb3dgs_oracle import *  # noqa: F401,F403
from . import mb3dgs_adc as adc  # noqa: F401
