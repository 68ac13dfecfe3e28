"""The seeded program generators: determinism and the workload shapes they promise."""
from workloads import (config1_chain6, config2_sc_grid, config3_ion_alltoall, config4_neutral_batch,
                       config5_spin_chain, program_stats)
from workloads.circuits import OP_NAMES, grid_edges


def test_generators_are_deterministic():
    for f in (config1_chain6, config2_sc_grid, config3_ion_alltoall, config5_spin_chain):
        assert f().ops == f().ops
    assert [p.ops for p in config4_neutral_batch(count=4)] == [p.ops for p in config4_neutral_batch(count=4)]
    assert config1_chain6(seed=1).ops != config1_chain6(seed=2).ops


def test_workload_shapes():
    p = config1_chain6()
    assert p.n == 6 and p.n_gates == 200
    p = config2_sc_grid()
    assert p.n == 14
    st = program_stats(p)
    assert st["by_name"]["zx"] == 15 * (6 + 6 + 4 + 3)      # 60 layers cycling over 4 edge classes
    assert st["by_name"]["bitflip"] == 14
    assert sum(len(c) for c in grid_edges(2, 7)) == 19
    p = config3_ion_alltoall()
    assert p.n == 15 and p.n_gates == 800
    p = config5_spin_chain()
    assert p.n == 16 and p.n_gates == 2000
    b = config4_neutral_batch(count=64)
    assert all(6 <= q.n <= 12 for q in b) and len({q.n for q in b}) > 3


def test_programs_use_known_ops_with_valid_qubits():
    for p in (config1_chain6(), config2_sc_grid(depth=4), config3_ion_alltoall(n_gates=50), config5_spin_chain(n_gates=60)):
        for o in p.ops:
            assert o.name in OP_NAMES
            assert len(set(o.qubits)) == len(o.qubits)
            assert all(0 <= q < p.n for q in o.qubits)
