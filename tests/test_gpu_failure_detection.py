"""Failure detection of the persistent kernels' bounded grid barrier, without a GPU
fault: a cooperative launch whose barrier waits for one more block than the launch has
(an arrival that nothing makes) must give up after its run-time limit, return
IGA_ERR_TIMEOUT, and leave the context usable."""
import numpy as np
import pytest

import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2004_05197_gb300 import iga
    from paper_2004_05197_gb300 import workloads as W


def test_barrier_opens_when_every_block_arrives():
    assert iga.iga_barrier_selftest(8, 8, 1000.0) == iga.IGA_OK


def test_barrier_wait_runs_out_and_context_stays_usable():
    assert iga.iga_barrier_selftest(8, 9, 1.0) == iga.IGA_ERR_TIMEOUT
    assert "ran out" in iga.iga_last_error()
    # the device still runs work: an FP64 apply against the same apply's second run
    w = W.scaled("annulus64_p2", n_el=12)
    sp = W.make_space(w)
    ops = iga.iga_surrogate_assemble(sp, w["p"], w["q"], w["M"])
    N = iga.iga_ops_info_get(ops).N
    x = torch.tensor(inputs.vectors(N, 1), device="cuda")
    y1, y2 = torch.empty_like(x), torch.empty_like(x)
    iga.iga_stencil_apply(ops, iga.IGA_OP_M, iga.IGA_F64, x, y1, 1)
    assert iga.iga_barrier_selftest(4, 4, 1000.0) == iga.IGA_OK
    iga.iga_stencil_apply(ops, iga.IGA_OP_M, iga.IGA_F64, x, y2, 1)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2) and float(y1.abs().max()) > 0.0
    iga.iga_ops_destroy(ops)
    iga.iga_space_destroy(sp)


def test_barrier_selftest_rejects_bad_arguments():
    for args in ((0, 1, 1.0), (1, 0, 1.0), (1, 1, 0.0), (100000, 1, 1.0)):
        with pytest.raises(iga.IgaError):
            iga.iga_barrier_selftest(*args)
