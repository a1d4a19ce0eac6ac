"""Sliding super point estimation (SRE/RSRA + SLE/SLEA) on B300.

Importing the package loads nothing native; ``paper_1805_09246_b300.sse`` binds the
CUDA library ``libsse.so`` on first use, and ``paper_1805_09246_b300.synth`` is the
seeded synthetic traffic generator.
"""
