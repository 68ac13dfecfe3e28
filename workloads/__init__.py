"""Seeded synthetic device programs (inputs shared by the oracle and the CUDA path).

This package holds no arithmetic of the emulation method: it only draws
random angles, device parameters and circuit layouts and emits them as
*native operations* ``(name, qubits, params)``.  Turning a native operation
into a unitary or a Kraus set is the device compiler's job, and each side
(oracle and library) implements that on its own.
"""
from .circuits import (NativeOp, Program, config1_chain6, config2_sc_grid, config3_ion_alltoall,
                       config4_neutral_batch, config5_spin_chain, OP_NAMES, program_stats)

__all__ = ["NativeOp", "Program", "config1_chain6", "config2_sc_grid", "config3_ion_alltoall",
           "config4_neutral_batch", "config5_spin_chain", "OP_NAMES", "program_stats"]
