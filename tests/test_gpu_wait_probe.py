"""Failure detection of the tensor-core kernels' bounded waits, without a fault or a hang.

Every mbarrier wait of the BF16 path's tcgen05 kernels gives up after a cycle
limit and reports the timeout status instead of hanging the GPU.  The probe runs
that same wait on a barrier that nothing arrives at, with a short limit: the
wait must end, report the timeout bit (128) to the host, and leave the context
usable (a tensor-core matvec right after it still matches its float64
reference); with an arrival first the same wait succeeds.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2503_00253_gb300 import binding
    binding.library()
    return binding


def test_bounded_wait_runs_out_and_reports_timeout(B):
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    B.wait_probe(1 << 22, False, status)          # about 2 ms at 2 GHz; nothing arrives
    torch.cuda.synchronize()
    assert int(status.item()) == 128
    B.wait_probe(1 << 22, True, status)           # the barrier's one arrival comes first
    torch.cuda.synchronize()
    assert int(status.item()) == 0


def test_context_usable_after_a_timed_out_wait(B):
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.wait_probe(1 << 20, False, status)
    torch.cuda.synchronize()
    assert int(status.item()) == 128
    # one row tile, two stored blocks, 20 systems: the product against its float64 reference
    g = torch.Generator(device="cuda").manual_seed(3)
    nrt, J = 1, 20
    rowptr = torch.tensor([0, 2], dtype=torch.int32, device="cuda")
    colblk = torch.tensor([0, 1], dtype=torch.int32, device="cuda")
    C = torch.randn((2, 128, 64), device="cuda", generator=g)
    C_hi = C.to(torch.bfloat16)
    C_lo = (C - C_hi.float()).to(torch.bfloat16)
    P = torch.randn((J, 128), device="cuda", generator=g).to(torch.bfloat16)
    sigma = torch.rand(J, device="cuda", generator=g) + 1.0
    Y, _, st = B.info_esrf_bf16_tile_matvec(rowptr, colblk, C_hi, C_lo, P, sigma)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    Cd = (C_hi.double() + C_lo.double())                      # [2][128][64]
    full = torch.cat([Cd[0], Cd[1]], dim=1)                   # rows of the tile x 128 columns
    ref = sigma.double()[:, None] * P.double() + (full @ P.double().T).T
    err = (Y.double() - ref).abs().max().item() / ref.abs().max().item()
    assert err < 1e-5, err


def test_wait_probe_rejects_bad_arguments(B):
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(B.InfoEsrfError) as e:
        B.wait_probe(0, False, status)
    assert e.value.code == B.ERR_INVALID_ARG
    with pytest.raises(B.InfoEsrfError):
        B.wait_probe((1 << 32) + 1, False, status)
