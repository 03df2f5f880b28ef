"""The BF16 block-tile matvec on the tensor cores (tcgen05, TMA-staged), through the C ABI.

y_j = sigma_j p_j + C p_j for J systems at once (App. E: the localized-covariance
product of every PCG iteration; C is shared by all systems, Sec. 2.3).  C is
given as 128 x 64 blocks in two BF16 planes (hi + lo); the products of BF16
numbers are exact in FP32, so the result must equal the float64 product of the
same BF16 values to FP32 accumulation accuracy.  Cases: ragged system counts in
both chunk widths (128, 256), row tiles with one block and with every block
(more blocks than pipeline stages), and the per-row-tile dot products p^T y.
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


def _random_blocks(rng, nrt, nblk):
    rowptr = [0]
    cols = []
    for t in range(nrt):
        k = [1, nblk, int(rng.integers(1, nblk + 1))][t % 3]
        c = np.sort(rng.choice(nblk, size=k, replace=False))
        cols.extend(c.tolist())
        rowptr.append(len(cols))
    return np.array(rowptr, dtype=np.int32), np.array(cols, dtype=np.int32)


@pytest.mark.parametrize("nrt,J", [(3, 50), (8, 300), (5, 128), (4, 257), (2, 1)])
def test_tile_matvec_matches_float64_product(B, nrt, J):
    rng = np.random.default_rng(nrt * 1000 + J)
    d_pad = 128 * nrt
    nblk = d_pad // 64
    rowptr, colblk = _random_blocks(rng, nrt, nblk)
    ntiles = colblk.size
    C = rng.standard_normal((ntiles, 128, 64)).astype(np.float32) * rng.uniform(0.1, 10.0, (ntiles, 128, 1))
    C_hi = torch.tensor(C).to(torch.bfloat16)
    C_lo = (torch.tensor(C) - C_hi.float()).to(torch.bfloat16)
    P = torch.tensor(rng.standard_normal((J, d_pad)).astype(np.float32)).to(torch.bfloat16)
    sigma = torch.tensor(rng.uniform(1.0, 50.0, J).astype(np.float32))
    Y, pty, status = B.info_esrf_bf16_tile_matvec(rowptr=torch.tensor(rowptr, device="cuda"),
                                                  colblk=torch.tensor(colblk, device="cuda"),
                                                  C_hi=C_hi.cuda(), C_lo=C_lo.cuda(), P=P.cuda(),
                                                  sigma=sigma.cuda())
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    # dense float64 reference of the same BF16 values
    Cd = np.zeros((d_pad, d_pad))
    Ce = C_hi.double().numpy() + C_lo.double().numpy()
    for t in range(nrt):
        for b in range(rowptr[t], rowptr[t + 1]):
            Cd[128 * t:128 * t + 128, 64 * colblk[b]:64 * colblk[b] + 64] = Ce[b]
    Pd = P.double().numpy()
    Yref = sigma.double().numpy()[:, None] * Pd + Pd @ Cd.T
    scale = np.abs(Pd) @ np.abs(Cd).T + np.abs(sigma.double().numpy()[:, None] * Pd)
    err = np.abs(Y.cpu().double().numpy() - Yref)
    assert np.all(err <= 1e-5 * scale + 1e-30), float(np.max(err / (scale + 1e-30)))
    ptyref = (Pd * Yref).reshape(J, nrt, 128).sum(-1).T
    ptyscale = (np.abs(Pd) * scale).reshape(J, nrt, 128).sum(-1).T
    assert np.all(np.abs(pty.cpu().double().numpy() - ptyref) <= 1e-5 * ptyscale + 1e-30)
