"""The BF16 block-tile path (tensor-core matvec) against the FP64 oracle, through the C ABI.

The analysis must match the oracle's same-node result (Sec. 3.2, exact
solves per node) within 1e-4 relative (the mixed-precision bound), element-wise
per member, at PCG tolerance 1e-6: a 1-D periodic problem (config-1 shape), a
reduced 2-D periodic shape of the 1024^2 configuration (128^2 grid,
observations every 2nd cell in each direction, Gaspari-Cohn half-width 12,
N = 16, Q = 8) against the sparse form of the oracle, a layered Lorenz-96
shape, and ragged or degenerate sizes (d not a multiple of 128, one
observation, two members, every point observed).
"""
import numpy as np
import pytest
import torch

from oracle import filter as F
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


def run(B, pr, tol=1e-6, **kw):
    opts = B.make_options(precision=B.PRECISION_BF16, **kw)
    mu_a, A_a, st = B.info_esrf_analysis(pr.grid, dev(pr.X), dev(pr.obs_idx), dev(pr.y), dev(pr.R), pr.Q, tol, opts)
    torch.cuda.synchronize()
    return mu_a.cpu().numpy(), A_a.cpu().numpy(), st


def check(pr, mu_a, A_a, sparse=False, bound=1e-4):
    if sparse:
        A_ref = S.perturbation_update(pr.X, pr.obs_idx, pr.R, pr.grid, pr.Q)
        mu_ref = S.mean_update(pr.X, pr.obs_idx, pr.y, pr.R, pr.grid)
    else:
        A_ref = F.perturbation_update(pr.X, pr.obs_idx, pr.R, pr.grid, pr.Q)
        mu_ref = F.mean_update(pr.X, pr.obs_idx, pr.y, pr.R, pr.grid)
    ea = increment_error(A_a, A_ref, pr.X - pr.X.mean(0))
    em = mean_error(mu_a, mu_ref, pr.X.mean(0))
    assert ea <= bound and em <= bound, (pr.name, ea, em)
    return ea, em


def test_bf16_config1_shape(B):
    pr = workloads.config1()
    mu_a, A_a, st = run(B, pr)
    assert st["status"] == 0 and st["solver_path"] == 3 and st["n_unconverged"] == 0, st
    ea, em = check(pr, mu_a, A_a)
    print(f"config1 BF16: {ea:.2e} {em:.2e}, iters {st['iters_mean']:.1f}/{st['iters_max']}")


def test_bf16_reduced_2d_matches_sparse_oracle(B):
    pr = workloads.gaussian_problem_2d(nx=128, ny=128, N=16, length_scale=8.0, obs_stride=2, r2=0.5,
                                       half_width=12.0, Q=8, tol=1e-6, seed=5)
    mu_a, A_a, st = run(B, pr)
    assert st["status"] == 0 and st["solver_path"] == 3 and st["n_unconverged"] == 0, st
    ea, em = check(pr, mu_a, A_a, sparse=True)
    print(f"2-D 128^2 BF16: {ea:.2e} {em:.2e}, iters {st['iters_mean']:.1f}/{st['iters_max']}")


def test_bf16_layered_l96(B):
    pr = workloads.layered_l96_problem(nx=240, nz=4, N=20, spinup=300, c_x=15.0, c_z=1.0, Q=12)
    mu_a, A_a, st = run(B, pr)
    assert st["status"] == 0 and st["n_unconverged"] == 0, st
    check(pr, mu_a, A_a)


@pytest.mark.parametrize("case", ["ragged", "one_obs", "two_members", "all_observed", "no_ritz", "ritz20"])
def test_bf16_ragged_and_degenerate_sizes(B, case):
    kw = {}
    if case == "ragged":
        pr = workloads.gaussian_problem_1d("rg", n=1000, N=12, length_scale=6.0, obs_stride=3, r2=0.4,
                                           half_width=9.0, Q=6, tol=1e-6, seed=3)      # d = 334
    elif case == "one_obs":
        pr = workloads.gaussian_problem_1d("one", n=64, N=8, length_scale=4.0, obs_stride=64, r2=0.5,
                                           half_width=5.0, Q=5, tol=1e-6, seed=4)      # d = 1
    elif case == "two_members":
        pr = workloads.gaussian_problem_1d("two", n=300, N=2, length_scale=5.0, obs_stride=2, r2=0.5,
                                           half_width=6.0, Q=7, tol=1e-6, seed=6)
    elif case == "all_observed":
        pr = workloads.gaussian_problem_1d("all", n=200, N=10, length_scale=5.0, obs_stride=1, r2=1.0,
                                           half_width=5.0, Q=6, tol=1e-6, seed=7)
    elif case == "no_ritz":
        pr = workloads.gaussian_problem_1d("nor", n=500, N=10, length_scale=5.0, obs_stride=2, r2=0.5,
                                           half_width=7.0, Q=6, tol=1e-6, seed=8)
        kw = dict(ritz_rank=0)
    else:   # more than 14 Ritz vectors: the 64-value dot-product path of the vector kernels
        pr = workloads.gaussian_problem_2d(nx=64, ny=64, N=12, length_scale=5.0, obs_stride=2, r2=0.5,
                                           half_width=6.0, Q=6, tol=1e-6, seed=9)
        kw = dict(ritz_rank=20, oversample=8)
    mu_a, A_a, st = run(B, pr, **kw)
    assert st["status"] == 0 and st["n_unconverged"] == 0, (case, st)
    check(pr, mu_a, A_a)


@pytest.mark.parametrize("N", [3, 17, 100, 128])
def test_bf16_member_counts(B, N):
    """Member counts around the 16-member steps of the tensor-core C formation and state update (the
    steps past N are skipped) and their largest case, N = 128, on a 2-D periodic grid."""
    pr = workloads.gaussian_problem_2d(nx=48, ny=48, N=N, length_scale=6.0, obs_stride=2, r2=0.5,
                                       half_width=5.0, Q=4, tol=1e-6, seed=40 + N)
    mu_a, A_a, st = run(B, pr)
    assert st["status"] == 0 and st["solver_path"] == 3 and st["n_unconverged"] == 0, (N, st)
    ea, em = check(pr, mu_a, A_a)
    print(f"N = {N}: {ea:.2e} {em:.2e}")


def test_bf16_matches_fp32_path_and_reports_unsupported(B):
    pr = workloads.gaussian_problem_1d("cmp", n=4096, N=24, length_scale=32.0, obs_stride=4, r2=0.25,
                                       half_width=128.0, Q=12, tol=1e-6, seed=9)
    mu16, A16, st16 = run(B, pr)
    o32 = B.make_options(precision=B.PRECISION_FP32)
    mu32, A32, st32 = B.info_esrf_analysis(pr.grid, dev(pr.X), dev(pr.obs_idx), dev(pr.y), dev(pr.R), pr.Q, 1e-6, o32)
    torch.cuda.synchronize()
    assert increment_error(A16, A32.cpu().numpy(), pr.X - pr.X.mean(0)) <= 1e-4
    print(f"iterations BF16 {st16['iters_mean']:.2f}/{st16['iters_max']}, FP32 {st32['iters_mean']:.2f}/{st32['iters_max']}")
    # multi-shift CG and more than 128 members are not taken by the BF16 path
    with pytest.raises(B.InfoEsrfError) as e:
        B.info_esrf_analysis(pr.grid, dev(pr.X), dev(pr.obs_idx), dev(pr.y), dev(pr.R), pr.Q, 1e-6,
                             B.make_options(precision=B.PRECISION_BF16, solver=B.SOLVER_MULTISHIFT))
    assert e.value.code == B.ERR_UNSUPPORTED
