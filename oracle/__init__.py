"""Oracle: a plain, slow, FP64 CPU restatement of the density-matrix emulation.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The
library and its Python binding never import it, and it imports nothing from
them; the two share only the seeded program generators in ``workloads/``.

Modules
-------
``compile``  device compiler: native operation -> unitary or Kraus set (Sec. 3, 4-8, App. B).
``evolve``   state initialisation and the literal update rho <- sum_k K rho K^dagger.
``measure``  probabilities, Pauli expectation values, trace, purity.
``brute``    independent full-space constructions (Kronecker chains, 4^n superoperators)
             used only to pin the oracle itself.

Parity status: every function here is pinned by tests in ``tests/test_oracle_pins.py``
except the readings listed as "parity unpinned" in their docstrings (none at present).
"""
from . import compile, evolve, measure, brute  # noqa: F401
