"""Independent CPU oracle for the per-shot sampler.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, link or
execute anything in this package; only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

The oracle shares no code with the CUDA path.  It is written from the paper
(Tsim, arXiv 2604.01059) and split into two independent halves:

* program semantics -- ``circuit`` (own Stim-subset parser and raw noise
  channel enumeration), ``statevector`` (exact branching state vector over
  Z[w, 1/sqrt2]) and ``frame`` (Pauli-frame flip propagation for Clifford
  circuits).  These say what probability a compiled program must produce.
* sampling semantics -- ``evaluator.c`` (plain C: its own program-file
  reader, its own Philox4x32-10, the phase-pair formula evaluated in exact
  Z[w] integer arithmetic, Algorithm 1 with the exact Bernoulli rule, and
  record packing), wrapped by ``evaluator`` (ctypes).

Every function cites the passage of the paper it follows.  Pins that tie
each part to something other than itself live in ``tests/test_oracle_*.py``.
"""
