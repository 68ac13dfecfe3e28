"""vqd_prob_static: the allocation-free probability reduction.

Some callers cannot allocate device memory (their framework's pool owns the GPU, or their loop must
not pay for the synchronisation cudaMalloc can cause).  vqd_prob_static serves them with partial sums
in a static device array.  Here it must give vqd_prob's result on two calls in a row (the array keeps
the previous call's contents), and refuse more measured qubits than its scratch allows.  This file is
collected last so that a failure here comes after every other test has run.
"""
import numpy as np
import pytest

from workloads import config2_sc_grid
from workloads.circuits import random_program

from ._lib import get_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vqd():
    return get_lib()


@pytest.mark.parametrize("prec_name", ["f64", "f32"])
def test_prob_static_matches_prob_twice(vqd, prec_name):
    torch = pytest.importorskip("torch")
    prec = vqd.VQD_F64 if prec_name == "f64" else vqd.VQD_F32
    stream = torch.cuda.current_stream().cuda_stream
    for n, prog, subsets in (
        (6, random_program(5, 6, 80), ([0], [5, 2], [3, 1, 4], list(range(6)))),
        (14, config2_sc_grid(depth=2), ([0], [13, 0, 7], list(range(14)))),
    ):
        ctx = vqd.vqd_create(n, prec, stream)
        try:
            vqd.vqd_apply_native(ctx, 0, prog.ops)
            for qs in subsets:
                want = vqd.vqd_prob(ctx, 0, qs)
                for _ in range(2):
                    out = torch.full((2 ** len(qs),), float("nan"), dtype=torch.float64, device="cuda")
                    vqd.vqd_prob_static(vqd.vqd_state_ptr(ctx, 0), n, prec, qs, out.data_ptr(), stream)
                    torch.cuda.current_stream().synchronize()
                    got = out.cpu().numpy()
                    assert np.abs(got - want).max() < 1e-13, (n, qs)
        finally:
            vqd.vqd_destroy(ctx)


def test_prob_static_rejects_more_qubits_than_its_scratch(vqd):
    torch = pytest.importorskip("torch")
    n = 15
    ctx = vqd.vqd_create(n, vqd.VQD_F32)
    try:
        out = torch.zeros(2 ** 15, dtype=torch.float64, device="cuda")
        with pytest.raises(vqd.VQDError) as e:
            vqd.vqd_prob_static(vqd.vqd_state_ptr(ctx, 0), n, vqd.VQD_F32, list(range(15)), out.data_ptr())
        assert e.value.code == vqd.VQD_EINVAL
        assert "14" in str(e.value)
        # the largest allowed request still works after the refusal
        vqd.vqd_prob_static(vqd.vqd_state_ptr(ctx, 0), n, vqd.VQD_F32, list(range(14)), out.data_ptr())
        torch.cuda.synchronize()
        got = out[: 2 ** 14].cpu().numpy()
        want = vqd.vqd_prob(ctx, 0, list(range(14)))
        assert np.abs(got - want).max() < 1e-13
        assert abs(got[0] - 1.0) < 1e-12          # |0><0| on 15 qubits: all weight on the all-zero outcome
    finally:
        vqd.vqd_destroy(ctx)
