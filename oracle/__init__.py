"""FP64 CPU oracle for the DiaQ gate-apply path (arXiv 2405.01250).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this package. The
product library never imports, links or runs it, and it never imports the
product. See ``oracle.core`` for what each function computes.
"""

from .core import *  # noqa: F401,F403
