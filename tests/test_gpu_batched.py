"""The batched uneven workload (many independent problems in one call, Sec. 3.3).

- Parity at the workload's largest sizes: the problem of largest n and the
  problem with the widest observation band of the 64-problem batch, in one
  batched call with two small problems, against the sparse form of the
  oracle's same-node result (exact solves per node, Sec. 3.2), at FP64
  (1e-10) and FP32 (1e-4), element-wise per member.
- The batched call captured in a CUDA graph and replayed equals the direct
  call bit for bit (FP64).
"""
import numpy as np
import pytest
import torch

from oracle import sparse as S
from paper_2503_00253_gb300 import workloads
from parity_checks import increment_error, mean_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2503_00253_gb300 import binding
    binding.library()
    return binding


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


def _dicts(B, probs, tol):
    out = []
    for p in probs:
        obs = dev(p.obs_idx)
        mo, mx = B.neighbor_counts(p.grid, obs)
        out.append(dict(grid=p.grid, X=dev(p.X), obs_idx=obs, y=dev(p.y), R=dev(p.R), Q=p.Q, tol=tol,
                        max_oo=mo, max_xo=mx))
    return out


@pytest.fixture(scope="module")
def large_subset():
    probs = workloads.uneven_batch(64)
    i_big = max(range(64), key=lambda i: probs[i].n)
    i_wide = min(range(64), key=lambda i: (probs[i].n / probs[i].d, -probs[i].d))
    small = sorted(range(64), key=lambda i: probs[i].n)[:2]
    chosen = [probs[i] for i in [i_big, i_wide] + small]
    refs = [(S.mean_update(p.X, p.obs_idx, p.y, p.R, p.grid), S.perturbation_update(p.X, p.obs_idx, p.R, p.grid, p.Q))
            for p in chosen]
    return chosen, refs


@pytest.mark.parametrize("precision,tol,bound", [(0, 1e-12, 1e-10), (1, 1e-6, 1e-4)])
def test_batched_largest_n_and_widest_band_match_sparse_oracle(B, large_subset, precision, tol, bound):
    probs, refs = large_subset
    assert max(p.n for p in probs) > 50000 and min(p.n / p.d for p in probs) < 4.5
    outs, stats = B.info_esrf_analysis_batched(_dicts(B, probs, tol), B.make_options(precision=precision))
    torch.cuda.synchronize()
    for p, (mu_a, A_a), st, (mu_ref, A_ref) in zip(probs, outs, stats, refs):
        assert st["status"] == 0 and st["n_unconverged"] == 0, (p.name, st)
        ea = increment_error(A_a, A_ref, p.X - p.X.mean(0))
        em = mean_error(mu_a, mu_ref, p.X.mean(0))
        assert ea <= bound and em <= bound, (p.name, precision, ea, em)


def test_batched_call_captured_in_a_cuda_graph(B):
    probs = workloads.uneven_batch(count=5, seed=12, tol=1e-12, n_min=300, n_max=3000)
    dicts = _dicts(B, probs, 1e-12)
    opts = B.make_options(precision=0)
    outs_direct, _ = B.info_esrf_analysis_batched(dicts, opts)
    torch.cuda.synchronize()
    ref = [(m.clone(), a.clone()) for m, a in outs_direct]
    for d, (m, a) in zip(dicts, outs_direct):
        d["mu_a"], d["A_a"] = m, a
        m.fill_(float("nan"))
        a.fill_(float("nan"))
    import ctypes
    arr = (B.ProblemC * len(dicts))()
    for i, d in enumerate(dicts):
        B._fill_problem(arr[i], d, d["X"], d["mu_a"], d["A_a"])
    need = B.library().info_esrf_batched_workspace_size(arr, len(dicts), ctypes.byref(opts))
    ws = B.workspace(need)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        B.info_esrf_analysis_batched(dicts, opts, ws=ws, stats=False, stream=stream)
    torch.cuda.synchronize()
    for rep in range(2):
        for d in dicts:
            d["mu_a"].fill_(float("nan"))
            d["A_a"].fill_(float("nan"))
        graph.replay()
        torch.cuda.synchronize()
        for d, (m, a) in zip(dicts, ref):
            assert torch.equal(d["mu_a"], m) and torch.equal(d["A_a"], a), rep
