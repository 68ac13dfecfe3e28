"""Oracle: a plain, slow, FP64 CPU restatement of the density-matrix emulation.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The
library and its Python binding never import it, and it imports nothing from
them; the two share only the seeded program generators in ``workloads/``.

Modules
-------
``compile``  device compiler: native operation -> unitary or Kraus set (Sec. 3, 4-8, App. B).
``evolve``   state initialisation and the literal update rho <- sum_k K rho K^dagger.
``cloop``    the same update as plain FP64 C loops (``c/kraus_loop.c``, gcc + OpenMP), for full-size runs
             and for the timed CPU baseline.
``measure``  probabilities, Pauli expectation values, trace, purity, trace distance, Uhlmann
             fidelity, projective and parity measurement with collapse (Secs. 6, 7).
``brute``    independent full-space constructions (Kronecker chains, 4^n superoperators)
             used only to pin the oracle itself.
``trajectories``  statevector trajectories with their own counter-based Philox draws (Sec. 2).
``schedule`` ASAP scheduling with passive idle noise (Sec. 2).
``devices``  the five device-family compilers (Secs. 4-8, App. C).

Parity status: every function here is pinned by tests in ``tests/test_oracle_pins.py``,
``tests/test_devices.py``, ``tests/test_trajectories.py`` and ``tests/test_abi_cpu.py``
(closed forms, worked examples, brute force), except the readings listed as "parity unpinned"
in their docstrings (none at present).
"""
from . import compile, evolve, measure, brute  # noqa: F401
