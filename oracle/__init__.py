"""CPU oracle for the depth-fused LBP + SVM hot path (arXiv 1504.01883).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  The
product path (``paper_1504_01883_gb300``) never imports it, and it never
imports the product path.  The only code both sides share is the seeded input
generator module ``paper_1504_01883_gb300.synth``, which holds no arithmetic
of the method.
"""
from .oracle import *  # noqa: F401,F403
