#!/usr/bin/env python
"""Benchmark: InFo-ESRF analyses per second on one GB300 (or N replicas).

One step = one full analysis (mean update + perturbation update: anomalies,
localized-covariance bands, quadrature, Ritz pairs, the persistent batched
shifted PCG over all 1280 + 1 systems, quadrature accumulation and the
state update) of the 1-D Gaussian-forecast workload n=8192, N=40, d=1024,
Q=32, in FP32 bulk arithmetic with FP64 scalars, through the C ABI.  By
default the shifted systems use the learned preconditioner correction,
trained before the timed region on three other seeds of the same workload;
the paper's preconditioner alone (FP32) and the FP64 path are timed beside it.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "perturbation-update analyses/sec at <=1e-4 rel err vs FP64; matvec HBM GB/s"
UNIT = "analyses/s"
WORKLOAD = "gauss1d_n8192_N40_d1024_Q32_R0.25_gc256 (1280 shifted systems + mean)"
TOL_MIXED = 1e-6
RITZ = 10
TRAIN_SEEDS = (11, 12, 13)
SOLVER_KERNELS = {0: "k_pcg (general persistent batched PCG)", 1: "k_pcg_band1d (cluster-resident band PCG)",
                  2: "k_mscg (multi-shift CG)", 3: "k_tile_mm + k_tpcg_* (BF16 tensor-core block-tile PCG)",
                  4: "k_bcg_* (block CG across members)"}
# DRAM bytes (read + write) of one launch of a kernel on the headline workload,
# measured by ncu (dram__bytes_read.sum + dram__bytes_write.sum) on this
# bench, keyed by the SHA-256 prefix of the kernel's source file when the
# counters were taken.  The figure is reported only while that file is
# unchanged; otherwise the line's "traffic" is null.
TRAFFIC = {
    "k_pcg_band1d": ("pcg_cluster.cu", "50caed7ddd104ac7", 1477376),
    "k_mscg": ("mscg.cu", "1fdc47a794982019", 1351680),
}


def _source_sha16(name):
    import hashlib
    path = os.path.join(ROOT, "paper_2503_00253_gb300", "csrc", name)
    with open(path, "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def _traffic(kernel):
    src, sha, nbytes = TRAFFIC[kernel]
    if sha is None or nbytes is None:
        return None
    return nbytes if _source_sha16(src) == sha else None


def _dist():
    from paper_2503_00253_gb300 import replicas
    return replicas.rank_info()


def _clock_sampler(path):
    cmd = ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
           "--format=csv,noheader,nounits", "-lms", "200"]
    try:
        return subprocess.Popen(cmd, stdout=open(path, "w"), stderr=subprocess.DEVNULL)
    except OSError:
        return None


def _clock_summary(path, gpu_index):
    sm, mx, reasons = [], 0.0, set()
    try:
        for line in open(path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9 or f[0] != str(gpu_index):
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
    except OSError:
        pass
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _oracle_analysis(pr):
    from oracle import filter as F
    mu = F.mean_update(pr.X, pr.obs_idx, pr.y, pr.R, pr.grid)
    A = F.perturbation_update(pr.X, pr.obs_idx, pr.R, pr.grid, pr.Q)
    return mu, A


def run_reference(args):
    """Reference arm: the FP64 CPU oracle, as it stands, on the host cores."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from paper_2503_00253_gb300 import workloads
    pr = workloads.config2()
    for _ in range(args.warmup):
        _oracle_analysis(pr)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _oracle_analysis(pr)
    dt = time.perf_counter() - t0
    value = args.steps / dt
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "precision": "fp64 dense oracle"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "one full analysis (mean + perturbation update, dense FP64) per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_general_h(args):
    """Weighted-sum observation operators (non-subsampling H, Sec. 2.3 model-space localization), the
    paper's two shapes: 100 Gaussian channel sums (b = 10) of a 2000-point circle, N = 20, Q = 16 (the
    single-cycle experiment's operator, Sec. 4.1); and 8 columns x 5 weighted vertical sums (b = 8,
    spacing 6) of a 40 x 32 layered grid, N = 40, Q = 8, localization length 3 (Sec. 5.1).  FP32 (tol
    1e-6) and FP64 (tol 1e-12); per case one untimed call, then `steps` direct calls of
    info_esrf_analysis_batched timed with the library's phase events, the fastest kept; the relative
    error against the FP64 oracle and the oracle's time on the host (untimed checks).  One JSON line
    per case."""
    import numpy as np
    import torch

    from oracle import filter as F
    from paper_2503_00253_gb300 import binding as B
    from paper_2503_00253_gb300 import workloads

    _, rank, local = _dist()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.library()
    cases = []
    pr = workloads.gaussian_problem_1d("chan", n=2000, N=20, length_scale=10.0, obs_stride=20, r2=0.5,
                                       half_width=20.0, Q=16, tol=1e-6, seed=91)
    H = workloads.gaussian_channel_operator(pr.n, 100, 10.0)
    R = np.full(100, 0.5)
    y = H[0] @ pr.truth + np.sqrt(R) * np.random.default_rng(92).standard_normal(100)
    cases.append(("gauss1d n2000 N20, 100 Gaussian channels b=10, Q16", pr, H, y, R))
    grid = workloads.Grid((40, 1, 32), (True, False, False), (3.0, 1.0, 3.0))
    base = workloads.random_obs_problem(grid, N=40, d=10, r2=0.25, Q=8, tol=1e-6, seed=93)
    H2 = workloads.column_sum_operator((40, 1, 32), list(range(0, 40, 5)), 5, 6.0, 8.0)
    R2 = np.full(40, 0.25)
    y2 = H2[0] @ base.truth + np.sqrt(R2) * np.random.default_rng(94).standard_normal(40)
    cases.append(("layered 40x32 N40, 8 columns x 5 channels, Q8", base, H2, y2, R2))
    stream = torch.cuda.current_stream(dev)
    for name, prb, Hc, yc, Rc in cases:
        t0 = time.perf_counter()
        A_ref = F.perturbation_update_H(prb.X, Hc[0], Rc, prb.grid, prb.Q)
        mu_ref = F.mean_update_H(prb.X, Hc[0], yc, Rc, prb.grid)
        oracle_s = time.perf_counter() - t0
        _, (rowptr, col, val) = Hc
        for prec, tol in ((B.PRECISION_FP32, TOL_MIXED), (B.PRECISION_FP64, 1e-12)):
            d = dict(grid=prb.grid, X=torch.tensor(prb.X, device=dev),
                     H=(torch.tensor(rowptr, device=dev), torch.tensor(col, device=dev),
                        torch.tensor(val, device=dev)),
                     y=torch.tensor(yc, device=dev), R=torch.tensor(Rc, device=dev), Q=prb.Q, tol=tol)
            opts = B.make_options(precision=prec)
            events = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
            for e in events:
                e.record(stream)
            B.set_phase_events(opts, events)
            outs, stats = B.info_esrf_analysis_batched([d], opts, stream=stream)
            torch.cuda.synchronize()
            best = None
            for _ in range(max(args.steps, 1)):
                outs, stats = B.info_esrf_analysis_batched([d], opts, stream=stream)
                events[4].synchronize()
                ph = [events[i].elapsed_time(events[i + 1]) for i in range(4)]
                tot = events[0].elapsed_time(events[4])
                if best is None or tot < best[0]:
                    best = (tot, ph)
            B.set_phase_events(opts, None)
            (mu_a, A_a), st = outs[0], stats[0]
            ea = F.relative_increment_error(A_a.cpu().numpy(), A_ref, prb.X - prb.X.mean(0))
            em = float(np.linalg.norm(mu_a.cpu().numpy() - mu_ref) / np.linalg.norm(mu_ref - prb.X.mean(0)))
            print(json.dumps({"workload": "general_h", "case": name, "precision": "fp32" if prec == 1 else "fp64",
                              "ms_per_analysis": best[0], "analyses_per_s": 1e3 / best[0],
                              "phases_ms": dict(zip(["setup", "ritz", "pcg", "finish"], best[1])),
                              "iters_mean": st["iters_mean"], "status": st["status"],
                              "solver_path": st["solver_path"], "rel_err": ea, "rel_err_mean": em,
                              "oracle_host_s": oracle_s}), flush=True)


def run_band_phases(args):
    """Per-round phase cycles of the 1-D band PCG kernel, and per-stage cycles of the fused eigensolver
    kernel, on the headline workload (learned model trained as
    in the default line, autotuned), from the instrumented build of the library (INFO_ESRF_PHASE_CLOCKS=1,
    set before the library loads). The timed bench line never uses the instrumented library."""
    os.environ["INFO_ESRF_PHASE_CLOCKS"] = "1"
    import torch

    from paper_2503_00253_gb300 import binding as B
    from paper_2503_00253_gb300 import learned, workloads

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    B.library()
    pr = workloads.config2()
    X, obs, y, R = (torch.tensor(a, device=dev) for a in (pr.X, pr.obs_idx, pr.y, pr.R))
    max_oo, max_xo = B.neighbor_counts(pr.grid, obs)
    theta, cutoff = None, 0.0
    if args.preconditioner == "learned":
        train_set = [workloads.config2(tol=TOL_MIXED, seed=s) for s in TRAIN_SEEDS]
        theta, cutoff, _ = learned.fit(train_set, K=12, members_per_q=3, steps=300)
    opts = B.make_options(precision=B.PRECISION_FP32, ritz_rank=RITZ, max_neighbors=max(max_oo, max_xo),
                          learned_model=theta, learned_max_shift=cutoff)
    if args.autotune:
        B.autotune([dict(grid=pr.grid, X=X, obs_idx=obs, y=y, R=R, Q=pr.Q, tol=TOL_MIXED, max_oo=max_oo,
                         max_xo=max_xo)], opts)
    st = None
    for _ in range(args.warmup):
        st = B.info_esrf_analysis(pr.grid, X, obs, y, R, pr.Q, TOL_MIXED, opts)[2]
    torch.cuda.synchronize()
    B.band_phase_clocks(reset=True)
    B.ritz_phase_clocks(reset=True)
    for _ in range(args.steps):
        B.info_esrf_analysis(pr.grid, X, obs, y, R, pr.Q, TOL_MIXED, opts)
    torch.cuda.synchronize()
    ph = B.band_phase_clocks(reset=True)
    ph["ritz"] = B.ritz_phase_clocks(reset=True)
    ph["launches"] = args.steps
    ph["ctas"] //= args.steps
    rec = {"workload": WORKLOAD, "kind": "band_phase_clocks", "preconditioner": args.preconditioner,
           "cluster_size": int(opts.cluster_size), "solver_path": st["solver_path"] if st else None,
           "iters_mean": st["iters_mean"] if st else None, **ph}
    print(json.dumps(rec))


def run_ours(args):
    import numpy as np
    import torch

    from paper_2503_00253_gb300 import binding as B
    from paper_2503_00253_gb300 import replicas, workloads

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    B.library()
    pr = workloads.config2()
    X = torch.tensor(pr.X, device=dev)
    obs = torch.tensor(pr.obs_idx, device=dev)
    y = torch.tensor(pr.y, device=dev)
    R = torch.tensor(pr.R, device=dev)
    N, n = pr.X.shape
    d = pr.d
    max_oo, max_xo = B.neighbor_counts(pr.grid, obs)
    cap = max(max_oo, max_xo)
    prec = B.PRECISION_FP32 if args.precision == "fp32" else B.PRECISION_FP64
    tol = TOL_MIXED if prec == B.PRECISION_FP32 else args.fp64_tol
    multishift = args.solver == "multishift"
    use_learned = args.preconditioner == "learned" and prec == B.PRECISION_FP32 and not multishift
    theta, cutoff, learn_info = None, 0.0, None
    if use_learned:
        from paper_2503_00253_gb300 import learned
        t0 = time.perf_counter()
        train_set = [workloads.config2(tol=TOL_MIXED, seed=s) for s in TRAIN_SEEDS]
        theta, cutoff, hist = learned.fit(train_set, K=12, members_per_q=3, steps=300)
        torch.cuda.synchronize()
        learn_info = {"train_seeds": list(TRAIN_SEEDS), "fit_s": time.perf_counter() - t0,
                      "loss_first": float(hist[0]), "loss_last": float(hist[-1]), "max_shift": cutoff}
    opts = B.make_options(precision=prec, ritz_rank=RITZ, max_neighbors=cap, learned_model=theta,
                          learned_max_shift=cutoff,
                          solver=B.SOLVER_MULTISHIFT if multishift else B.SOLVER_PCG)
    # native autotuner (untimed): cluster size, power iterations and oversampling of the eigensolver,
    # the settings that do not change the converged answer
    tune_info = None
    if args.autotune and not multishift:
        t0 = time.perf_counter()
        best = B.autotune([dict(grid=pr.grid, X=X, obs_idx=obs, y=y, R=R, Q=pr.Q, tol=tol, max_oo=max_oo,
                                max_xo=max_xo)], opts)
        torch.cuda.synchronize()
        tune_info = {"cluster_size": int(opts.cluster_size), "power_iters": int(opts.power_iters),
                     "oversample": int(opts.oversample), "best_ms": best, "tune_s": time.perf_counter() - t0}
    g = B.make_grid(pr.grid)
    import ctypes
    need = B.library().info_esrf_workspace_size(ctypes.byref(g), N, d, pr.Q, ctypes.byref(opts))
    wsp = B.workspace(need, dev)
    mu_a = torch.empty(n, dtype=torch.float64, device=dev)
    A_a = torch.empty((N, n), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(stats=False):
        return B.info_esrf_analysis(pr.grid, X, obs, y, R, pr.Q, tol, opts, ws=wsp, mu_a=mu_a, A_a=A_a,
                                    stats=stats, stream=stream)[2]

    # one run with stats: iteration counts for the flop count, and parity vs the oracle
    st = step(stats=True)
    torch.cuda.synchronize()
    result = {}
    ref_cache = None
    if rank == 0 and not args.no_parity:
        from oracle import filter as F
        mu_ref, A_ref = _oracle_analysis(pr)
        ref_cache = (mu_ref, A_ref)
        Af = pr.X - pr.X.mean(0)
        result["rel_err"] = F.relative_increment_error(A_a.cpu().numpy(), A_ref, Af)
        mu0 = pr.X.mean(0)
        result["rel_err_mean"] = float(np.linalg.norm(mu_a.cpu().numpy() - mu_ref) / np.linalg.norm(mu_ref - mu0))

    # exact band size and per-system iteration counts for the algorithmic flop count
    prep = B.Prepared(pr.grid, X, obs, R, pr.Q, B.make_options(precision=prec, ritz_rank=RITZ, max_neighbors=cap,
                                                              oversample=int(opts.oversample),
                                                              power_iters=int(opts.power_iters)))
    nnz_C = int(prep.export("oo_nnz").sum())
    del prep
    it_sys = torch.zeros(1 + pr.Q * N, dtype=torch.int32, device=dev)
    o_it = B.make_options(precision=prec, ritz_rank=RITZ, max_neighbors=cap, learned_model=theta,
                          learned_max_shift=cutoff, system_iters=it_sys, oversample=int(opts.oversample),
                          power_iters=int(opts.power_iters), solver=int(opts.solver))
    o_it.cluster_size = opts.cluster_size
    B.info_esrf_analysis(pr.grid, X, obs, y, R, pr.Q, tol, o_it, ws=wsp, mu_a=mu_a, A_a=A_a, stats=False,
                         stream=stream)
    it_sys = it_sys.cpu().numpy().astype(np.float64)
    s_nodes, _ = B.info_esrf_quadrature_nodes(pr.Q, st["ell_used"])
    sigma_sys = np.concatenate([[1.0], np.repeat(s_nodes.cpu().numpy() + 1.0, N)])
    learned_sys = (sigma_sys <= cutoff) if use_learned else np.zeros_like(sigma_sys, dtype=bool)

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    events = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    for e in events:
        e.record(stream)
    B.set_phase_events(opts, events)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # CUDA graph of one analysis call (the library's launch sequence, replayed
    # without host launch overhead); the direct call is the fallback
    graph, graph_err, graph_launches = None, None, 0
    if args.graph:
        B.set_phase_events(opts, None)           # timing events cannot be recorded inside a graph
        try:
            cap_stream = torch.cuda.Stream(dev)
            cap_stream.wait_stream(stream)
            g_ = torch.cuda.CUDAGraph()
            n_cap0 = B.launch_count()
            with torch.cuda.graph(g_, stream=cap_stream):
                B.info_esrf_analysis(pr.grid, X, obs, y, R, pr.Q, tol, opts, ws=wsp, mu_a=mu_a, A_a=A_a,
                                     stats=False, stream=cap_stream)
            stream.wait_stream(cap_stream)
            graph_launches = B.launch_count() - n_cap0
            graph = g_
            for _ in range(args.warmup):
                with torch.cuda.stream(stream):
                    graph.replay()
            torch.cuda.synchronize()
        except Exception as exc:                  # capture refused: time the direct call
            graph, graph_err = None, f"{type(exc).__name__}: {exc}"
            torch.cuda.synchronize()

    def timed_step():
        if graph is not None:
            with torch.cuda.stream(stream):
                graph.replay()
        else:
            step()

    clock_path = os.path.join(tempfile.gettempdir(), f"clocks_{os.getpid()}.csv")
    sampler = _clock_sampler(clock_path) if rank == 0 else None
    time.sleep(0.3 if sampler else 0.0)
    replicas.barrier()
    torch.cuda.synchronize()
    launches0 = B.launch_count()
    step_ms = []
    t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for s in range(args.steps):
        flush.fill_(float(s))                       # evicts L2 between timed steps
        t0e.record(stream)
        timed_step()
        t1e.record(stream)
        t1e.synchronize()
        step_ms.append(t0e.elapsed_time(t1e))
    torch.cuda.synchronize()
    launches = B.launch_count() - launches0
    if graph is not None:
        launches = graph_launches * args.steps      # kernels in the graph, replayed once per step
    total_ms = replicas.max_over_ranks(sum(step_ms), dev)
    replicas.barrier()
    # phase times (and the PCG launch time of the roofline) from direct calls
    # with events recorded at the phase boundaries
    B.set_phase_events(opts, events)
    pcg_ms, phase_ms = [], []
    for s in range(max(3, min(args.steps, 10))):
        flush.fill_(float(s))
        step()
        events[4].synchronize()
        phase_ms.append([events[i].elapsed_time(events[i + 1]) for i in range(4)])
        pcg_ms.append(phase_ms[-1][2])
    B.set_phase_events(opts, None)

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    Xh = torch.tensor(pr.X).pin_memory()
    obsh = torch.tensor(pr.obs_idx).pin_memory()
    yh = torch.tensor(pr.y).pin_memory()
    Rh = torch.tensor(pr.R).pin_memory()
    mu_h = torch.empty(n, dtype=torch.float64).pin_memory()
    A_h = torch.empty((N, n), dtype=torch.float64).pin_memory()
    Xd, obsd, yd, Rd = (torch.empty_like(t, device=dev) for t in (Xh, obsh, yh, Rh))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_ms = []
    for s in range(args.warmup + args.steps):
        flush.fill_(float(s))
        e0.record(stream)
        for dst, src in ((Xd, Xh), (obsd, obsh), (yd, yh), (Rd, Rh)):
            dst.copy_(src, non_blocking=True)
        B.info_esrf_analysis(pr.grid, Xd, obsd, yd, Rd, pr.Q, tol, opts, ws=wsp, mu_a=mu_a, A_a=A_a,
                             stats=False, stream=stream)
        mu_h.copy_(mu_a, non_blocking=True)
        A_h.copy_(A_a, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        if s >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    if sampler:
        sampler.terminate()
        sampler.wait()
    clocks = _clock_summary(clock_path, local) if rank == 0 else {}
    h2d = sum(t.numel() * t.element_size() for t in (Xh, obsh, yh, Rh))
    d2h = mu_h.numel() * 8 + A_h.numel() * 8
    e2e_total = replicas.max_over_ranks(sum(e2e_ms), dev)

    # comparators on the same GPU: the paper's preconditioner alone, in FP32 and in FP64
    comparators = {}
    if rank == 0 and prec == B.PRECISION_FP32 and args.fp64_steps > 0:
        cases = [("fp64_pcg", B.PRECISION_FP64, B.SOLVER_PCG)]
        if use_learned or multishift:
            cases.insert(0, ("lmp_fp32", B.PRECISION_FP32, B.SOLVER_PCG))
        if not multishift:
            # one unpreconditioned CG run per member for all shifts (Sec. 3.3)
            cases.insert(0, ("multishift_fp32", B.PRECISION_FP32, B.SOLVER_MULTISHIFT))
            # block CG across members, one block per node (Sec. 3.3, second alternative)
            cases.insert(1, ("block_fp32", B.PRECISION_FP32, B.SOLVER_BLOCK))
        for key, pc, sv in cases:
            # the headline's autotuned eigensolver settings, so that only the
            # preconditioner (or the solver, or the precision) differs
            oc = B.make_options(precision=pc, ritz_rank=RITZ, max_neighbors=cap, solver=sv,
                                oversample=int(opts.oversample), power_iters=int(opts.power_iters))
            if sv == B.SOLVER_PCG:
                oc.cluster_size = opts.cluster_size
            needc = B.library().info_esrf_workspace_size(ctypes.byref(g), N, d, pr.Q, ctypes.byref(oc))
            wc = B.workspace(needc, dev)
            muc = torch.empty_like(mu_a)
            Ac = torch.empty_like(A_a)
            stc = B.info_esrf_analysis(pr.grid, X, obs, y, R, pr.Q, TOL_MIXED, oc, ws=wc, mu_a=muc, A_a=Ac,
                                       stats=True, stream=stream)[2]
            phc = []
            B.set_phase_events(oc, events)
            for s in range(args.fp64_steps):
                flush.fill_(float(s))
                B.info_esrf_analysis(pr.grid, X, obs, y, R, pr.Q, TOL_MIXED, oc, ws=wc, mu_a=muc, A_a=Ac,
                                     stats=False, stream=stream)
                events[4].synchronize()
                phc.append([events[i].elapsed_time(events[i + 1]) for i in range(4)])
            B.set_phase_events(oc, None)
            # timed like the headline: CUDA-graph replays of the analysis call
            # (direct calls where capture is refused), L2 flushed between steps
            gc, how = None, "direct call"
            # the block solver tests convergence on the host every iteration: not capturable
            if args.graph and sv != B.SOLVER_BLOCK:
                try:
                    cs_ = torch.cuda.Stream(dev)
                    cs_.wait_stream(stream)
                    gc = torch.cuda.CUDAGraph()
                    with torch.cuda.graph(gc, stream=cs_):
                        B.info_esrf_analysis(pr.grid, X, obs, y, R, pr.Q, TOL_MIXED, oc, ws=wc, mu_a=muc, A_a=Ac,
                                             stats=False, stream=cs_)
                    stream.wait_stream(cs_)
                    torch.cuda.synchronize()
                    how = "cuda graph of the analysis call"
                except Exception:
                    gc = None
                    torch.cuda.synchronize()
            ts = []
            for s in range(args.fp64_steps):
                flush.fill_(float(s))
                e0.record(stream)
                if gc is not None:
                    with torch.cuda.stream(stream):
                        gc.replay()
                else:
                    B.info_esrf_analysis(pr.grid, X, obs, y, R, pr.Q, TOL_MIXED, oc, ws=wc, mu_a=muc, A_a=Ac,
                                         stats=False, stream=stream)
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            del gc
            comparators[key] = {"value": 1e3 / statistics.mean(ts), "unit": UNIT, "tol": TOL_MIXED,
                                "solver_path": stc["solver_path"], "kernel": SOLVER_KERNELS[stc["solver_path"]],
                                "oversample": int(oc.oversample), "power_iters": int(oc.power_iters),
                                "steps": args.fp64_steps, "iters_mean": stc["iters_mean"],
                                "iters_max": stc["iters_max"], "ms_per_step": statistics.mean(ts),
                                "phases_ms": [statistics.mean(p[i] for p in phc) for i in range(4)],
                                "launch": how}
            if "rel_err" in result:
                from oracle import filter as F
                mu_ref, A_ref = ref_cache
                comparators[key]["rel_err"] = F.relative_increment_error(Ac.cpu().numpy(), A_ref,
                                                                        pr.X - pr.X.mean(0))
            del wc

    # FMA probe: measured FP32 ALU rate of this GPU (context for the ALU roofline)
    probe32, _ = B.fma_probe(1, 1 << 16)

    if rank != 0:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    ms_step = total_ms / args.steps
    value = replicas.whole_job_rate(args.steps, ws, total_ms)
    # algorithmic work of the PCG launch, per row of one system-iteration:
    #   2 nnz(C)/d (matvec) + 2 (shift) + 8 k (LMP projections and apply) + 10 (dots, axpys),
    #   + 68 where the learned term is active (a z, 33-tap S^T S r, add)
    flops_row = 2 * nnz_C / d + 2 + 8 * RITZ + 10
    pcg_flops = d * float(np.sum(it_sys * (flops_row + 68.0 * learned_sys)))
    kernel = "k_pcg_band1d (cluster-resident persistent batched shifted PCG)"
    traffic = _traffic("k_pcg_band1d") if (prec == B.PRECISION_FP32 and use_learned) else None
    if multishift:
        # multi-shift CG: per iteration of a chain (one member, or the mean)
        # 2 nnz(C) + 2 d (matvec and base shift) + 8 d (r and p updates, two dots),
        # and per row of every active shift 5 (its direction and the weighted sum)
        chain_it = np.concatenate([[it_sys[0]], it_sys[1:].reshape(pr.Q, N).max(axis=0)])
        pcg_flops = float(np.sum(chain_it)) * (2.0 * nnz_C + 10.0 * d) + 5.0 * d * float(np.sum(it_sys))
        kernel = "k_mscg (cluster-resident multi-shift CG, one Krylov run per member for all shifts)"
        traffic = _traffic("k_mscg") if prec == B.PRECISION_FP32 else None
    pcg_ms_mean = statistics.mean(pcg_ms)
    achieved = pcg_flops / (pcg_ms_mean * 1e-3) / 1e12
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    max_mhz = clocks.get("sm_max_mhz") or 2070.0
    peak = sms * 128 * 2 * max_mhz * 1e6 / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if prec == B.PRECISION_FP32 else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "N": N, "d": d, "Q": pr.Q, "systems": st["n_systems"],
                   "precision": "fp32 bulk, fp64 scalars and quadrature sum" if prec else "fp64",
                   "preconditioner": ("none (multi-shift CG, Sec. 3.3)" if multishift else
                                      "LMP + learned correction" if use_learned else "LMP"),
                   "solver": args.solver,
                   "tol": tol, "ritz_rank": RITZ, "band_nnz": nnz_C, "l2": "flushed between steps (512 MB write)",
                   "replicas": ws, "launch": "cuda graph of the analysis call" if graph is not None else
                   "direct call", **({"graph_error": graph_err} if graph_err else {})},
        "clocks": clocks,
        "e2e": {"value": replicas.whole_job_rate(args.steps, ws, e2e_total), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "kernel": kernel,
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": traffic, "peak_source": f"{sms} SMs x 128 FP32 lanes x 2 x {max_mhz:.0f} MHz",
                     "fma_probe_tflops": probe32 / 1e12, "pcg_ms": pcg_ms_mean,
                     "flops_per_launch": pcg_flops},
        "matvec_hbm_gbs": (traffic / (pcg_ms_mean * 1e-3) / 1e9) if traffic else None,
        "direct_call_ms": statistics.mean(sum(p) for p in phase_ms),
        "phases_ms": {k: statistics.mean(p[i] for p in phase_ms)
                      for i, k in enumerate(["setup_a1_a3", "ritz_a4", "pcg_a5_a8", "finish_a9_a11"])},
        "iters_mean": st["iters_mean"], "iters_max": st["iters_max"], "ell": st["ell_used"],
    }
    line.update(result)
    line.update(comparators)
    if not args.no_config5:
        # the 2-D workload on the BF16 tensor-core path, its own record (one warm-up, two timed analyses)
        line["config5"] = config5_record(B, dev, steps=2, warmup=1, no_parity=args.no_parity,
                                         learned_term=not args.no_config5_learned)
    if learn_info:
        line["learned"] = learn_info
    if tune_info:
        line["autotune"] = tune_info
    if not args.no_cpu_baseline:
        from oracle import filter as F  # noqa: F401
        t0 = time.perf_counter()
        runs = 0
        while runs < 3 and (time.perf_counter() - t0) < 20.0:
            _oracle_analysis(pr)
            runs += 1
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": runs / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"{runs} full analyses of the same workload (dense FP64 NumPy/LAPACK)"}
    print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


SMALL_2D = {"nx": 512, "half_width": 48.0, "Q": 8}   # profiling case of the 2-D family: a few GB on the device


def config5_record(B, dev, steps, warmup, no_parity=False, ritz=RITZ, learned_term=True, small=False):
    """The 2-D workload at full size: periodic 1024 x 1024 grid (n = 1,048,576), N = 80 from a
    Gaussian covariance with length scale 32 cells, observations every 2nd cell in each direction
    (d = 262,144), R = 0.5, Gaspari-Cohn half-width 96 cells, Q = 32 (2560 + 1 systems), on the BF16
    block-tile path (tensor-core matvec), tol 1e-6.  Direct calls timed with CUDA events (the path
    synchronizes once per PCG iteration, so it is not captured in a graph); inputs and workspace
    (about 70 GB) are far larger than L2.  The roofline is that of the tensor-core matvec: algorithmic
    FLOPs 2 nnz(C) + 2 d per system-iteration over the summed device time of its launches, against
    the measured sustained BF16 tensor peak.

    Learned correction (learned_term): the 2-D lattice form, trained before the timed region on
    Krylov samples of the BF16 path from two problems of the same geometry on a 512 x 512 grid
    (seeds 51, 52; 12 directions of 3 members per node, 300 Adam steps), with the shift cut-off
    chosen by the plain-PCG comparison on those problems; the timed analyses use it where that comparison
    keeps it.

    small: the same family on a 512 x 512 grid with GC half-width 48 cells and Q = 8 (d = 65,536,
    641 systems, about 3 GB of C blocks), the case that ncu captures of the path's kernels use."""
    import numpy as np
    import torch

    from paper_2503_00253_gb300 import learned, workloads
    learn_info, theta, cutoff = None, None, 0.0
    if learned_term:
        t0 = time.perf_counter()
        train = [workloads.gaussian_problem_2d(nx=512, ny=512, N=80, length_scale=32.0, obs_stride=2, r2=0.5,
                                               half_width=96.0, Q=32, tol=TOL_MIXED, seed=s) for s in (51, 52)]
        theta, cutoff, hist = learned.fit_lattice(train, K=12, members_per_q=3, steps=300)
        torch.cuda.synchronize()
        learn_info = {"train": "2 problems of the same geometry on 512 x 512 (seeds 51, 52), BF16-path "
                               "Krylov samples, 300 Adam steps", "fit_s": time.perf_counter() - t0,
                      "loss_first": float(hist[0]), "loss_last": float(hist[-1]), "max_shift": cutoff}
        del train
    t0 = time.perf_counter()
    if small:
        pr = workloads.gaussian_problem_2d(nx=SMALL_2D["nx"], ny=SMALL_2D["nx"], N=80, length_scale=32.0,
                                           obs_stride=2, r2=0.5, half_width=SMALL_2D["half_width"],
                                           Q=SMALL_2D["Q"], tol=TOL_MIXED, seed=5)
        label = "gauss2d_{0}x{0}_N80_d{1}_Q{2}_R0.5_gc{3:g} ({4} shifted systems + mean)".format(
            SMALL_2D["nx"], pr.d, SMALL_2D["Q"], SMALL_2D["half_width"], SMALL_2D["Q"] * 80)
    else:
        pr = workloads.config5(tol=TOL_MIXED)
        label = "gauss2d_1024x1024_N80_d262144_Q32_R0.5_gc96 (2560 shifted systems + mean)"
    gen_s = time.perf_counter() - t0
    X = torch.tensor(pr.X, device=dev)
    obs = torch.tensor(pr.obs_idx, device=dev)
    y = torch.tensor(pr.y, device=dev)
    R = torch.tensor(pr.R, device=dev)
    N, n = pr.X.shape
    it_sys = torch.zeros(1 + pr.Q * N, dtype=torch.int32, device=dev)
    opts = B.make_options(precision=B.PRECISION_BF16, ritz_rank=ritz, oversample=min(10, 32 - ritz),
                          system_iters=it_sys, learned_model=theta, learned_max_shift=cutoff)
    import ctypes
    g = B.make_grid(pr.grid)
    need = B.library().info_esrf_workspace_size(ctypes.byref(g), N, pr.d, pr.Q, ctypes.byref(opts))
    wsp = B.workspace(need, dev)
    mu_a = torch.empty(n, dtype=torch.float64, device=dev)
    A_a = torch.empty((N, n), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    events = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    for e in events:
        e.record(stream)           # torch creates the CUDA event at its first record
    B.set_phase_events(opts, events)
    times, stats, phases = [], [], []
    for s_ in range(warmup + steps):
        e0.record(stream)
        st = B.info_esrf_analysis(pr.grid, X, obs, y, R, pr.Q, TOL_MIXED, opts, ws=wsp, mu_a=mu_a, A_a=A_a,
                                  stats=True, stream=stream)[2]
        e1.record(stream)
        e1.synchronize()
        if s_ >= warmup:
            times.append(e0.elapsed_time(e1))
            stats.append(st)
            phases.append([events[i].elapsed_time(events[i + 1]) for i in range(4)])
    B.set_phase_events(opts, None)
    its = it_sys.cpu().numpy().astype(np.float64)
    st = stats[-1]
    flops = float(np.sum(its)) * (2.0 * st["c_nnz"] + 2.0 * pr.d)
    mm_ms = statistics.mean(x["matvec_ms"] for x in stats)
    peaks = _measured_peaks()
    peak = peaks.get("bf16_tflops_sustained")
    achieved = flops / (mm_ms * 1e-3) / 1e12
    issued_per_alg = (st["tile_blocks"] * 128 * 64 * 2.0) / st["c_nnz"]
    rec = {"workload": label,
           "precision": "bf16 tensor-core matvec (C as hi + lo BF16 planes, BF16 directions), fp32 vectors, "
                        "fp64 scalars and quadrature sum",
           "value": 1e3 / statistics.mean(times), "unit": UNIT, "ms_per_step": statistics.mean(times),
           "steps": steps, "warmup": warmup, "launch": "direct calls (one stream sync per PCG iteration)",
           "tol": TOL_MIXED, "ritz_rank": ritz, "iters_mean": st["iters_mean"], "iters_max": st["iters_max"],
           "n_unconverged": st["n_unconverged"], "status": st["status"], "solver_path": st["solver_path"],
           "c_nnz": st["c_nnz"], "taps_per_row": st["c_nnz"] / pr.d, "tile_blocks": st["tile_blocks"],
           "workspace_gb": need / 1e9, "input_gen_s": gen_s, "ell": st["ell_used"], "gershgorin": st["gershgorin"],
           "phases_ms": {k: statistics.mean(p[i] for p in phases)
                         for i, k in enumerate(["setup_a1_a3", "ritz_a4", "pcg_a5_a8", "finish_a9_a11"])},
           "iters_hist": np.histogram(its, bins=[0, 10, 20, 40, 80, 160, 320, 640, 2000])[0].tolist(),
           "learned": learn_info, "learned_stats": st["learned"],
           "roofline": {"bound": "tensor", "kernel": "k_tile_mm (tcgen05.mma kind::f16, TMA-staged)",
                        "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                        "frac": (achieved / peak) if peak else None,
                        "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (measured)",
                        "traffic": None, "matvec_ms_per_analysis": mm_ms,
                        "matvec_launches": stats[-1]["matvec_launches"], "flops_per_analysis": flops,
                        "issued_tensor_flops_per_algorithmic": issued_per_alg,
                        "issued_tensor_tflops": achieved * issued_per_alg}}
    if not no_parity:
        # at this size the oracle cannot form the update; a property that holds at any size:
        # the analysis perturbations keep zero ensemble mean (Thm. 3, linearity of the solves)
        A = A_a.cpu().numpy()
        Af = pr.X - pr.X.mean(0)
        rec["zero_mean_rel"] = float(np.max(np.abs(A.sum(0))) / np.max(np.abs(A - Af)))
    del wsp
    torch.cuda.empty_cache()
    return rec


def run_config5(args):
    import torch

    from paper_2503_00253_gb300 import binding as B
    _, rank, local = _dist()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.library()
    small = args.workload == "gauss2d_512"
    rec = config5_record(B, dev, args.steps, args.warmup, args.no_parity, args.ritz,
                         learned_term=not args.no_config5_learned and not small, small=small)
    line = {"metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": rec["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": rec["workload"], "precision": rec["precision"], "launch": rec["launch"],
                       "l2": "inputs and workspace far larger than L2"},
            "roofline": rec["roofline"], "config5": rec}
    print(json.dumps(line), flush=True)


def run_tilemm(args):
    """The tensor-core block-tile matvec alone (stage entry info_esrf_bf16_tile_matvec), on a seeded
    synthetic block structure with the 2-D workload's shape per row tile: 256 row tiles of 128
    observations (d_pad = 32,768), 300 stored 128 x 64 blocks per row tile (hi + lo BF16 planes),
    J = 2561 systems (161 units of 16, 11 chunks of at most 16 units).  About 3 GB on the device,
    more than L2.  Timed with CUDA events per launch after warm-up; FLOPs counted as issued by the
    tensor cores (two planes, 2 x 128 x 64 x 16 per block and unit)."""
    import numpy as np
    import torch

    from paper_2503_00253_gb300 import binding as B
    _, rank, local = _dist()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.library()
    nrt, per_row, J = 256, 300, 2561
    nblk = 2 * nrt
    rng = np.random.default_rng(17)
    cols = np.stack([np.sort(rng.choice(nblk, size=per_row, replace=False)) for _ in range(nrt)])
    rowptr = torch.tensor(np.arange(nrt + 1) * per_row, dtype=torch.int32, device=dev)
    colblk = torch.tensor(cols.reshape(-1), dtype=torch.int32, device=dev)
    ntiles = nrt * per_row
    gen = torch.Generator(device=dev).manual_seed(5)
    C = torch.randn((ntiles, 128, 64), device=dev, generator=gen)
    C_hi = C.to(torch.bfloat16)
    C_lo = (C - C_hi.float()).to(torch.bfloat16)
    del C
    torch.cuda.empty_cache()
    P = torch.randn((J, 128 * nrt), device=dev, generator=gen).to(torch.bfloat16)
    sigma = torch.rand(J, device=dev, generator=gen) + 1.0
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        B.info_esrf_bf16_tile_matvec(rowptr, colblk, C_hi, C_lo, P, sigma, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ts = []
    for _ in range(args.steps):
        e0.record(stream)
        _, _, status = B.info_esrf_bf16_tile_matvec(rowptr, colblk, C_hi, C_lo, P, sigma, stream=stream)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    assert int(status.item()) == 0
    units = (J + 15) // 16
    flops = ntiles * units * 2 * 2.0 * 128 * 64 * 16
    nbytes = ntiles * 2 * 16384 + 2.0 * J * 128 * nrt + 4.0 * J * 128 * nrt
    ms = statistics.mean(ts)
    peaks = _measured_peaks()
    peak = peaks.get("bf16_tflops")
    line = {"metric": "tensor-core block-tile matvec TFLOP/s (issued)", "value": flops / (ms * 1e-3) / 1e12,
            "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": f"tilemm: {nrt} row tiles x {per_row} blocks, J={J}", "ntiles": ntiles},
            "roofline": {"bound": "tensor", "achieved": flops / (ms * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                         "frac": (flops / (ms * 1e-3) / 1e12 / peak) if peak else None,
                         "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst, measured)",
                         "min_bytes": nbytes, "min_bytes_gbs": nbytes / (ms * 1e-3) / 1e9}}
    print(json.dumps(line), flush=True)


def run_batched(args):
    """Config-4 workload: 64 independent uneven 1-D problems (n log-uniform in [1024, 65536], N in
    {20, 40, 80}, observation stride 4..16, Q 16..48, seed 4) as one batched call (one launch per
    stage, one persistent PCG or multi-shift launch over all systems), against the same 64 problems
    as 64 single calls.  Both are captured as CUDA graphs and replayed with L2 flushed between steps;
    one step analyses all 64 problems.  Parity: the batched FP32 result against the batched FP64 one
    (every problem), and the problems with n <= 3000 against the dense FP64 oracle."""
    import numpy as np
    import torch

    from paper_2503_00253_gb300 import binding as B
    from paper_2503_00253_gb300 import workloads

    _, rank, local = _dist()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.library()
    probs = workloads.uneven_batch(64)
    prec = B.PRECISION_FP32 if args.precision == "fp32" else B.PRECISION_FP64
    tol = TOL_MIXED if prec == B.PRECISION_FP32 else args.fp64_tol
    solver = B.SOLVER_MULTISHIFT if args.solver == "multishift" else B.SOLVER_PCG
    dicts = []
    for p in probs:
        obs = torch.tensor(p.obs_idx, device=dev)
        mo, mx = B.neighbor_counts(p.grid, obs)
        dicts.append(dict(grid=p.grid, X=torch.tensor(p.X, device=dev), obs_idx=obs,
                          y=torch.tensor(p.y, device=dev), R=torch.tensor(p.R, device=dev), Q=p.Q, tol=tol,
                          max_oo=mo, max_xo=mx,
                          mu_a=torch.empty(p.n, dtype=torch.float64, device=dev),
                          A_a=torch.empty((p.N, p.n), dtype=torch.float64, device=dev)))
    opts = B.make_options(precision=prec, solver=solver)
    stream = torch.cuda.current_stream(dev)
    _, stats = B.info_esrf_analysis_batched(dicts, opts, stream=stream)
    torch.cuda.synchronize()
    import ctypes
    arr = (B.ProblemC * len(dicts))()
    for i, dd in enumerate(dicts):
        B._fill_problem(arr[i], dd, dd["X"], dd["mu_a"], dd["A_a"])
    wsb = B.workspace(B.library().info_esrf_batched_workspace_size(arr, len(dicts), ctypes.byref(opts)), dev)
    singles = []
    for p, dd in zip(probs, dicts):
        g = B.make_grid(p.grid)
        o1 = B.make_options(precision=prec, solver=solver, max_neighbors=max(dd["max_oo"], dd["max_xo"]))
        need = B.library().info_esrf_workspace_size(ctypes.byref(g), p.N, p.d, p.Q, ctypes.byref(o1))
        singles.append((o1, B.workspace(need, dev), torch.empty_like(dd["mu_a"]), torch.empty_like(dd["A_a"])))

    def batched(st):
        B.info_esrf_analysis_batched(dicts, opts, ws=wsb, stats=False, stream=st)

    def sequential(st):
        for p, dd, (o1, w1, m1, a1) in zip(probs, dicts, singles):
            B.info_esrf_analysis(p.grid, dd["X"], dd["obs_idx"], dd["y"], dd["R"], p.Q, tol, o1, ws=w1, mu_a=m1,
                                 A_a=a1, stats=False, stream=st)

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {}
    for key, fn in (("batched", batched), ("sequential", sequential)):
        fn(stream)
        torch.cuda.synchronize()
        cs = torch.cuda.Stream(dev)
        cs.wait_stream(stream)
        graph = torch.cuda.CUDAGraph()
        n0 = B.launch_count()
        with torch.cuda.graph(graph, stream=cs):
            fn(cs)
        launches = B.launch_count() - n0
        stream.wait_stream(cs)
        for _ in range(args.warmup):
            with torch.cuda.stream(stream):
                graph.replay()
        torch.cuda.synchronize()
        ts = []
        for s_ in range(args.steps):
            flush.fill_(float(s_))
            e0.record(stream)
            with torch.cuda.stream(stream):
                graph.replay()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        res[key] = {"ms_per_step": statistics.mean(ts), "best_ms": min(ts),
                    "value": 64e3 / statistics.mean(ts), "gpu_launches_per_step": launches}
        del graph
    # parity: FP32 batched against FP64 batched (all), small problems against the dense oracle
    parity = {}
    if not args.no_parity:
        from oracle import filter as F
        o64 = B.make_options(precision=0, solver=solver)
        out64, _ = B.info_esrf_analysis_batched(
            [dict(dd, tol=args.fp64_tol, mu_a=None, A_a=None) for dd in dicts], o64)
        torch.cuda.synchronize()
        worst64 = 0.0
        worst_or = 0.0
        for p, dd, (m64, a64) in zip(probs, dicts, out64):
            Af = p.X - p.X.mean(0)
            worst64 = max(worst64, F.relative_increment_error(dd["A_a"].cpu().numpy(), a64.cpu().numpy(), Af))
            if p.n <= 3000:
                A_ref = F.perturbation_update(p.X, p.obs_idx, p.R, p.grid, p.Q)
                worst_or = max(worst_or, F.relative_increment_error(dd["A_a"].cpu().numpy(), A_ref, Af))
        parity = {"rel_err_vs_fp64_batched_max": worst64, "rel_err_vs_oracle_small_max": worst_or}
    its = [st["iters_mean"] for st in stats]
    line = {"metric": METRIC, "value": res["batched"]["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["batched"]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec else "f64", "data": "synthetic",
            "config": {"workload": "uneven64: 64 independent 1-D Gaussian-forecast problems, n log-uniform in "
                                   "[1024, 65536], N in {20, 40, 80}, obs stride 4..16, Q 16..48, seed 4",
                       "systems": int(sum(st["n_systems"] for st in stats)), "solver": args.solver, "tol": tol,
                       "l2": "flushed between steps (512 MB write)",
                       "launch": "cuda graph of one batched call vs cuda graph of 64 single calls"},
            "batched": res["batched"], "sequential": res["sequential"],
            "speedup_vs_sequential": res["sequential"]["ms_per_step"] / res["batched"]["ms_per_step"],
            "iters_mean_over_problems": statistics.mean(its), "unconverged": int(sum(st["n_unconverged"]
                                                                                     for st in stats))}
    line.update(parity)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--preconditioner", default="learned", choices=["learned", "lmp"])
    ap.add_argument("--solver", default="pcg", choices=["pcg", "multishift"],
                    help="pcg: one PCG run per shifted system (the headline); multishift: one CG run per member "
                         "for all shifts (Sec. 3.3)")
    ap.add_argument("--graph", type=int, default=1, help="replay the analysis as a CUDA graph (0: direct calls)")
    ap.add_argument("--autotune", type=int, default=1, help="run the native autotuner before the timed region")
    ap.add_argument("--fp64-tol", type=float, default=1e-12)
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-parity", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-config5", action="store_true", help="skip the 2-D BF16 record of the default line")
    ap.add_argument("--no-config5-learned", action="store_true",
                    help="2-D record without training the lattice form of the learned correction")
    ap.add_argument("--ritz", type=int, default=RITZ, help="Ritz rank of the preconditioner (config5)")
    ap.add_argument("--workload", default="config2",
                    choices=["config2", "batched64", "config5", "gauss2d_512", "tilemm", "band_phases",
                             "general_h"],
                    help="config2: the headline single analysis; batched64: 64 uneven problems in one batched "
                         "call against 64 single calls; gauss2d_512: the 2-D BF16 path on a 512 x 512 grid "
                         "(profiling case); band_phases: per-round phase cycles of the band PCG "
                         "kernel (instrumented build)")
    args = ap.parse_args()
    if args.warmup < 3 and args.workload not in ("config5", "gauss2d_512"):
        args.warmup = 3   # config5: one analysis takes seconds; --warmup as given (at least 1)
    args.warmup = max(args.warmup, 1)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched64":
        run_batched(args)
    elif args.workload in ("config5", "gauss2d_512"):
        run_config5(args)
    elif args.workload == "tilemm":
        run_tilemm(args)
    elif args.workload == "band_phases":
        run_band_phases(args)
    elif args.workload == "general_h":
        run_general_h(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
