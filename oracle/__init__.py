"""CPU oracle for the ProAICD progressive refactor / retrieve path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

It is a plain, slow, numpy restatement of the method of arXiv 2609.04573
("adaptive interpolation + coefficient decomposition", ProAICD), written step
by step from the paper (Sections IV-VI, Algorithms 1 and 2), with no blocking,
fusion or reordering beyond what those steps state.  It shares no code with
the CUDA library; the only shared module is ``synth`` (seeded inputs).

Modules
-------
geometry  levels, regions, decomposition sub-levels, stream lattices (Sec. IV, V-B, V-C)
interp    1-D predictors, per-level / per-region passes, coefficient
          decomposition and their inverses (Sec. IV, V-B, Alg. 1, Alg. 2)
bitplane  quantisation, generic / negabinary+XOR bitplanes, sign
          sub-streams, exact error statistics (Sec. V-C, VI-A table, VI-C)
bounds    error-bound composition, max ordering, greedy retrieval planner
          (Sec. III-A, V-C, VI-B)
pipeline  refactor() and retrieve() end to end (Alg. 1, Alg. 2)

Pins: every function here is checked in ``tests/test_oracle_*.py`` against
closed forms, brute force and invariants the paper fixes.  Functions without
such a pin are listed as "parity unpinned" in their docstrings.
"""
from .pipeline import refactor, retrieve, plan, Scheme, Target  # noqa: F401
