"""Benchmark of the GB300 RGDBEK solver (one JSON line on stdout).

Workload: the sparse inconsistent least-squares system of 200000 x 50000 with
20 distinct uniformly random columns per row, N(0,1) values, b = A x* + e,
e ~ N(0, 1e-4) (sigma 1e-2), solved by RGDBEK with eta = 0.1 for rows and
columns until ||A^T(b - Ax)|| / ||A^T b|| <= 1e-8 (the minimum-norm
least-squares solution).  A step is one full solve from x_0 = 0; the metric
is outer iterations per second over the K timed solves, with the matrix and
b resident in HBM; L2 is flushed (a 256 MiB write) before every timed solve.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload sparse_ls|batched_deblur|poisson_mixed|deblur_adjoint]

The default workload is the headline above.  The others measure the other
forms of the solver, one JSON line each, on one GPU:
  batched_deblur  256 blur systems of sides 64..512 (2.07e9 nonzeros in all),
                  a fixed budget of outer iterations each, in ONE batched
                  launch (team size from the tuner); against solving them one
                  after another with the whole GPU each
  poisson_mixed   the P1 Poisson system on 1024 x 1024 nodes (1.05e6
                  unknowns), a fixed budget, FP32 inner products against FP64
  deblur_adjoint  the implicit adjoint on the regularised 256 x 256 deblur
                  ([A; 0.05 I], 131072 x 65536), FP64 and FP32 inner products

--impl reference times the FP64 CPU oracle (the plain implementation of the
paper's Algorithm 1 used by the tests) on the same workload: the K timed steps
together run ONE full solve to the tolerance, cut into K pieces (each piece
resumes the previous one's x_k, z_k and iteration number, which the oracle
continues bit-identically), so the reported rate is that of the whole solve.
Under torchrun (N > 1) every rank solves its own independent system of the
same shape (seed + rank): no data-path collective, weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

WORKLOAD = dict(name="sparse_ls_200000x50000_k20", m=200000, n=50000, k=20, sigma=1e-2, seed=1,
                eta=0.1, tol=1e-8, stop_rule="normal_eq", max_iter=100000)
METRIC = "RGDBEK outer iterations/s (time-to-1e-8 normal-equation residual)"
UNIT = "iters/s"
L2_FLUSH_BYTES = 256 << 20
REF_TRAJECTORY_ITERS = 260     # --impl reference: the K steps cover this many iterations


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--max-iter", type=int, default=None,
                    help="cap on outer iterations per solve (profiling runs only)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-repeats", type=int, default=1,
                    help="full oracle solves timed for cpu_baseline (the median is reported)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--precision", choices=["fp64", "fp32"], default="fp64",
                    help="the timed solve: FP64 (headline) or the FP32 form (FP32 inner "
                         "iterations in FP64 refinement) to the same FP64 tolerance")
    ap.add_argument("--only-spmv-large", action="store_true",
                    help="print only the 2000000 x 500000 SpMV measurement (profiling)")
    ap.add_argument("--no-spmv-large", action="store_true",
                    help="skip the 2000000 x 500000 SpMV bandwidth measurement")
    ap.add_argument("--no-adaptive", action="store_true",
                    help="skip the secondary solve with the adaptive inner tolerance")
    ap.add_argument("--workload", default="sparse_ls",
                    choices=["sparse_ls", "batched_deblur", "poisson_mixed", "deblur_adjoint"])
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--budget", type=int, default=None,
                    help="outer iterations per system (batched_deblur, poisson_mixed)")
    ap.add_argument("--inner-max", type=int, default=None,
                    help="LSQR step cap per block solve (batched_deblur)")
    ap.add_argument("--col-team", type=int, default=None,
                    help="CTAs of the column team of the two-team schedule (0 automatic, -1 one "
                         "team); default: the library's automatic choice")
    ap.add_argument("--smem-kb", type=int, default=None,
                    help="dynamic shared memory per CTA of the solve kernel in KB (default: "
                         "the library's automatic size)")
    ap.add_argument("--fp32", action="store_true",
                    help="batched_deblur: the FP32 form (FP64 refinement) instead of FP64")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_system(rank: int):
    """The benchmark system of this rank (independent systems per rank)."""
    w = WORKLOAD
    return workloads.sparse_ls(w["m"], w["n"], w["k"], sigma=w["sigma"], seed=w["seed"] + rank)


def make_system_small(rank: int):
    """The same recipe at 2000 x 500 (for host-side tests)."""
    w = WORKLOAD
    return workloads.sparse_ls(2000, 500, w["k"], sigma=w["sigma"], seed=w["seed"] + rank)


# ---------------------------------------------------------------------------
# Algorithmic bytes of one solve (FP64 values, int32 indices, int64 pointers),
# from the per-iteration counters the kernel reports.  Compulsory traffic of
# each phase: matrix arrays streamed once per pass, each vector read or
# written once per phase that touches it.
# ---------------------------------------------------------------------------
def algorithmic_bytes(st, m: int, n: int, nnz: int) -> float:
    it = st.iters
    full_passes = it * ((12 * nnz + 16 * m + 56 * n)        # column pass (A^T z, A^T t, x = xt)
                        + (12 * nnz + 24 * m + 8 * n))      # residual pass t = b - A xt
    # the last column pass (the converged test) has no residual pass after it
    full_passes += 12 * nnz + 16 * m + 56 * n
    # quantise (weights read, prefix sums and marks written, the other side's
    # line counts cleared) and compaction (marks read, list written)
    selection = it * (22 * n + 22 * m) + 4 * (st.sum_nu + st.sum_nj)
    # extraction by scatter: the selected lines' pointers, and per block entry
    # its index and value read, the target line's pointer gathered, its count
    # incremented, index and value written
    extraction = 16 * (st.sum_nu + st.sum_nj) + 36 * (st.sum_nnz_u + st.sum_nnz_j)
    # each inner solve first copies both sides of its block into shared memory;
    # the scattered side is sorted there and written back and reread
    caching = 48 * st.sum_nnz_u + 48 * st.sum_nnz_j + 16 * it * (m + n)
    zstep = it * 52 * m + 12 * st.sum_nnz_u + 8 * st.sum_nu
    lsqr_u = 24 * st.lsqr_nnz_u + 32 * m * st.inner_u + 90 * st.lsqr_n_u
    lsqr_j = (12 * st.sum_nnz_j + 16 * n * it + 8 * st.sum_nj        # first v of each row block
              + 24 * st.lsqr_nnz_j + 88 * n * st.inner_j + 44 * st.lsqr_n_j)
    return float(full_passes + selection + extraction + caching + zstep + lsqr_u + lsqr_j)


def critical_phases(st, col_team: int) -> int:
    """Grid phases on the critical chain of one solve (see grid_phases)."""
    if col_team > 0:
        return 6 * st.iters + 2 * st.inner_j
    return 10 * st.iters + 2 * (st.inner_u + st.inner_j)


# FP64 flops of one solve: 2 per stored nonzero per sparse product (the
# vector updates are O(m + n) and left out).  Per outer iteration: A^T z and
# A^T t in the column pass, A xt in the residual pass; per inner solve: the
# first A_U^T z (or A^J-side product), two products per LSQR step, and the
# z update A_U y.
FP64_PEAK_TFLOPS = 1.25  # GB300 nominal dense FP64 (no FP64 tensor path)


def algorithmic_flops(st, nnz: int) -> float:
    it = st.iters
    full = 2 * nnz * (3 * it + 2)
    inner = 2 * (2 * st.lsqr_nnz_u + 2 * st.sum_nnz_u) + 2 * (2 * st.lsqr_nnz_j + st.sum_nnz_j)
    return float(full + inner)


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.out = None

    def start(self):
        try:
            import tempfile
            self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.seek(0)
        rows = [r.split(",") for r in self.out.read().strip().splitlines() if r.count(",") >= 8]
        self.out.close()
        try:
            os.remove(self.out.name)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if r[5 + i].strip().lower() == "active"})
        loaded = [v for v in sm if smax and v > 0.5 * max(smax)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------
def _oracle_options(max_iter: int, tol: float):
    import oracle
    w = WORKLOAD
    return oracle.Options(eta_col=w["eta"], eta_row=w["eta"], stop_rule=2, tol=tol,
                          inner_tol=1e-10, inner_max=200, max_iter=max_iter, seed=0)


def oracle_time_to_tol(S, repeats: int = 1):
    """The oracle's full solve of the benchmark system from x_0 = 0 to the
    benchmark tolerance (seed 0, eta 0.1, single thread), timed `repeats`
    times; returns (iterations, median seconds, all seconds, final normal
    residual)."""
    import oracle
    w = WORKLOAD
    times, res = [], None
    for _ in range(max(1, repeats)):
        t0 = time.perf_counter()
        res = oracle.solve(S.A, S.b, _oracle_options(w["max_iter"], w["tol"]), n=S.n)
        times.append(time.perf_counter() - t0)
    return res.iters, statistics.median(times), times, res.normal_res


def cpu_baseline_entry(S, repeats: int):
    it, t, times, nrm = oracle_time_to_tol(S, repeats)
    return {"value": it / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "time_to_tol_s": t, "iters": it, "final_normal_res": nrm,
            "runs_s": times, "host_cpus": os.cpu_count(),
            "sample": f"full solve of the same system from x_0 = 0 to normal-equation "
                      f"residual {WORKLOAD['tol']:g} (seed 0, eta {WORKLOAD['eta']}), FP64 C "
                      f"oracle on one thread, median of {len(times)}"}


def run_reference(args):
    """The oracle on the host: the K timed steps run one full solve to the
    tolerance cut into K pieces, each resuming the previous piece's state
    (bit-identical to one uninterrupted solve); warm-up steps run one
    iteration each."""
    import oracle
    rank, world, _ = dist_env()
    if rank != 0:
        return
    S = make_system(0)
    w = WORKLOAD
    for _ in range(args.warmup):
        oracle.solve(S.A, S.b, _oracle_options(1, w["tol"]), n=S.n)
    per = max(1, -(-REF_TRAJECTORY_ITERS // max(1, args.steps)))
    x, z, k = np.zeros(S.n), S.b.copy(), 0
    times, iters, done, nrm = [], 0, False, None
    for _ in range(args.steps):
        if done:
            times.append(0.0)
            continue
        t0 = time.perf_counter()
        part = oracle.solve(S.A, S.b, _oracle_options(k + per, w["tol"]), n=S.n,
                            resume=(x, z, k))
        times.append(time.perf_counter() - t0)
        iters += part.iters - k
        x, z, k = part.x, part.z, part.iters
        nrm = part.normal_res
        done = part.status == 0
    total = sum(times)
    value = iters / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": w["name"], "m": w["m"], "n": w["n"], "nnz": S.nnz,
                   "eta": w["eta"], "tol": w["tol"], "stop_rule": w["stop_rule"]},
        "time_to_tol_s": total if done else None, "iters": iters, "converged": done,
        "final_normal_res": nrm,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "host_cpus": os.cpu_count(),
                         "sample": f"one solve from x_0 = 0 to normal-equation residual "
                                   f"{w['tol']:g} (or {per * args.steps} iterations), cut into "
                                   f"{args.steps} resumed pieces of {per} iterations, FP64 C "
                                   f"oracle on one thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "_rgdbek_build", os.path.join(ROOT, "paper_2509_19267_gb300", "build.py"))
    bmod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bmod)
    if rank == 0:
        bmod.build()
    if dist is not None:
        dist.barrier()
    import paper_2509_19267_gb300 as rg

    w = WORKLOAD
    max_iter = args.max_iter if args.max_iter is not None else w["max_iter"]
    S = make_system(rank)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    opts = dict(eta_col=w["eta"], eta_row=w["eta"], stop_rule=rg.STOP_NORMAL)
    if args.col_team is not None:
        opts["col_team"] = args.col_team
    if args.smem_kb is not None:
        opts["smem_per_cta"] = 1024 * args.smem_kb
    if args.precision == "fp32":
        opts["precision"] = rg.PRECISION_FP32_INNER
    if args.only_spmv_large:
        peak, _ = measured_peaks()
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        print(json.dumps({"spmv_large": spmv_large(rg, dev, flush, peak)}), flush=True)
        return
    solver = rg.Solver(S.m, S.n, S.row_ptr, S.col_idx, S.vals, **opts)
    info = solver.info()
    b = torch.from_numpy(S.b).to(dev)
    x = torch.empty(S.n, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def one_solve(seed):
        st = rg.rgdbek_solve(solver.handle, b, x, w["tol"], max_iter, seed)
        return st

    for i in range(args.warmup):
        flush.fill_(float(i))
        one_solve(1000 + i)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    stats = []
    for i in range(args.steps):
        flush.fill_(float(i))                     # evict A and the vectors from L2
        ev[i][0].record(stream)
        stats.append(one_solve(i))
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    ms = [a.elapsed_time(bb) for a, bb in ev]
    total_s = sum(ms) / 1e3
    iters = sum(s.iters for s in stats)
    total_max, iters_all = aggregate(total_s, iters, dist, dev)
    value = iters_all / total_max

    # roofline of the dominant kernel (the persistent solve kernel): algorithmic
    # bytes per launch over its CUDA-event duration
    peak, peak_kind = measured_peaks()
    bytes_per = [algorithmic_bytes(s, S.m, S.n, S.nnz) for s in stats]
    achieved = sum(bytes_per) / total_s / 1e9
    flops_per = [algorithmic_flops(s, S.nnz) for s in stats]
    fp64_tflops = sum(flops_per) / total_s / 1e12
    # DRAM bytes per launch: ncu's dram__bytes_read + dram__bytes_write per outer
    # iteration of this kernel (from a short capture of the same system), times
    # the iterations of the timed solves; null once the kernel sources changed
    traffic = None
    tp = os.path.join(ROOT, "profiles", "solve_kernel_traffic.json")
    if os.path.exists(tp):
        with open(tp) as f:
            tj = json.load(f)
        if tj.get("kernel_source_hash") == source_hash():
            traffic = tj["dram_bytes_per_outer_iteration"] * iters / len(stats)

    # standalone SpMV kernels (the a1 / a5 products), L2 flushed before each launch
    spmv = spmv_rooflines(rg, solver, S, dev, flush, peak)
    spmv_big = None
    if not args.no_spmv_large and rank == 0:
        spmv_big = spmv_large(rg, dev, flush, peak)

    # secondary figure: the same solve with the inner tolerance tied to the
    # outer residual (inner_adapt = 0.1); the headline keeps the fixed one
    adaptive = None
    if not args.no_adaptive:
        adaptive = adaptive_inner(rg, S, opts, w, max_iter, b, x, flush, stream, args)

    # secondary figure: the same solve with FP32 inner products
    fp32 = None
    if not args.no_adaptive:
        fp32 = fp32_inner(rg, S, opts, w, max_iter, b, x, flush, stream, args)

    # secondary figure: eta chosen by the measured tuner, and the time to the
    # tolerance at every candidate (the headline keeps eta = 0.1)
    eta = None
    if not args.no_adaptive:
        eta = eta_tuning(rg, S, opts, w, max_iter, b, flush, stream)

    # end to end through the public API with host buffers: create from pinned
    # host CSR (H2D of A and the CSC/norm set-up), solve with host b and x
    e2e = None
    if not args.no_e2e:
        e2e = end_to_end(rg, S, opts, w, max_iter, args)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline_entry(S, args.cpu_repeats)

    if rank == 0:
        st0 = stats[0]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32 inner / f64 refinement",
            "data": "synthetic",
            "config": {"workload": w["name"], "m": S.m, "n": S.n, "nnz": S.nnz, "eta": w["eta"],
                       "tol": w["tol"], "stop_rule": w["stop_rule"],
                       "l2": "flushed before every timed solve (256 MiB write)",
                       "grid": info.grid, "threads_per_block": info.threads_per_block,
                       "col_team": info.col_team, "smem_per_cta": info.smem_per_cta,
                       "parallelism": "independent system per GPU" if world > 1 else "1 GPU"},
            "time_to_tol_s": statistics.median(ms) / 1e3,
            "iters_per_solve": [s.iters for s in stats],
            "final_normal_res": st0.normal_res, "final_rel_res": st0.rel_res,
            "per_iteration": {"lsqr_steps_col": st0.inner_u / max(st0.iters, 1),
                              "lsqr_steps_row": st0.inner_j / max(st0.iters, 1),
                              "block_cols": st0.sum_nu / max(st0.iters, 1),
                              "block_rows": st0.sum_nj / max(st0.iters, 1),
                              "nnz_A_U": st0.sum_nnz_u / max(st0.iters, 1),
                              "nnz_A_J": st0.sum_nnz_j / max(st0.iters, 1)},
            "phase_ms": {k: round(v, 3) for k, v in st0.as_dict()["phase_ms"].items()},
            "wall_s": wall,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "solve_kernel (persistent, one launch per solve)",
                         "peak_source": peak_kind,
                         "algorithmic_bytes_per_launch": statistics.mean(bytes_per),
                         "fp64": {"flops_per_launch": statistics.mean(flops_per),
                                  "achieved_tflops": fp64_tflops,
                                  "peak_tflops": FP64_PEAK_TFLOPS, "peak_source": "nominal",
                                  "frac": fp64_tflops / FP64_PEAK_TFLOPS}},
            # the solve is a chain of grid-synchronised phases.  One team: per
            # outer iteration 9 (two passes, two quantise and draw phases, two
            # compaction-scatters, z update) plus one for the row step's first
            # LSQR vector, and two per LSQR step.  Two teams: the row team's
            # chain, 6 per iteration (r phase, quantise, draws, scatter, first
            # vector, residual pass) and two per row LSQR step; the column
            # team's phases run beside it
            "grid_phases": {
                "chain": "row team" if info.col_team > 0 else "one team",
                "per_solve": critical_phases(st0, info.col_team),
                "us_per_phase": 1e6 * statistics.median(ms) / 1e3 / max(
                    1, critical_phases(st0, info.col_team))},
            "spmv": spmv,
            "spmv_large": spmv_big,
            "adaptive_inner": adaptive,
            "eta_tuning": eta,
            "fp32_inner": fp32,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": 2 * args.steps,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    solver.close()
    if dist is not None:
        dist.destroy_process_group()


def aggregate(total_s: float, iters: int, dist=None, device=None):
    """Whole-job numbers over the ranks: the slowest rank's timed seconds and
    the outer iterations of all ranks (each rank solved its own system)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(total_s), float(iters)
    import torch
    t = torch.tensor([total_s, float(iters)], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(t[1])


def source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2509_19267_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def spmv_rooflines(rg, solver, S, dev, flush, peak):
    import torch
    xv = torch.randn(S.n, dtype=torch.float64, device=dev)
    zv = torch.randn(S.m, dtype=torch.float64, device=dev)
    y = torch.empty(S.m, dtype=torch.float64, device=dev)
    g = torch.empty(S.n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    out = {}
    # algorithmic bytes: matrix (12 B/nnz + pointers) + source vector once + result once
    cases = {"csr_Ax": (lambda: rg.rgdbek_spmv(solver.handle, xv, y),
                        12 * S.nnz + 8 * (S.m + 1) + 8 * S.n + 8 * S.m),
             "csc_ATz": (lambda: rg.rgdbek_spmv_t(solver.handle, zv, g),
                         12 * S.nnz + 8 * (S.n + 1) + 8 * S.m + 8 * S.n)}
    for name, (fn, nbytes) in cases.items():
        for _ in range(3):
            fn()
        ts = []
        for i in range(20):
            a, bb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            # the flush (a 256 MiB write) evicts A from L2; the GPU-side delay
            # after it keeps the GPU busy while the host queues the start event
            # and the timed launch, so that no host launch latency is timed
            flush.fill_(float(i))
            torch.cuda._sleep(400000)
            a.record(stream)
            fn()
            bb.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(bb) / 1e3)
        t = statistics.median(ts)
        gbs = nbytes / t / 1e9
        out[name] = {"us": t * 1e6, "algorithmic_bytes": nbytes, "GB/s": gbs, "frac": gbs / peak}
    # context: a torch copy moving the same number of bytes (half read, half
    # written), timed the same way; the measured copy peak comes from a 4 GiB
    # copy, which a one-shot transfer of about 50 MB after an L2 flush cannot reach
    half = out["csr_Ax"]["algorithmic_bytes"] // 16
    src = torch.randn(half, dtype=torch.float64, device=dev)
    dst = torch.empty_like(src)
    ts = []
    for i in range(20):
        a, bb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(float(i))
        torch.cuda._sleep(400000)
        a.record(stream)
        dst.copy_(src)
        bb.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(bb) / 1e3)
    t = statistics.median(ts)
    out["same_size_copy"] = {"us": t * 1e6, "bytes": 16 * half, "GB/s": 16 * half / t / 1e9,
                             "frac": 16 * half / t / 1e9 / peak}
    for name in ("csr_Ax", "csc_ATz"):
        out[name]["frac_of_same_size_copy"] = out[name]["GB/s"] / out["same_size_copy"]["GB/s"]
    return out


SPMV_LARGE = dict(m=2000000, n=500000, k=20, seed=7)


def spmv_large(rg, dev, flush, peak):
    """The full-matrix products (a1 A^T z over the CSC copy, a5 A x over the
    CSR form) on the benchmark's recipe at 2000000 x 500000 (40M nonzeros,
    480 MB per copy of A: far larger than L2), after rgdbek_tune_spmv chose
    the lane split of each; L2 flushed before every timed launch."""
    import torch
    w = SPMV_LARGE
    t0 = time.perf_counter()
    S = workloads.sparse_ls(w["m"], w["n"], w["k"], sigma=1e-2, seed=w["seed"])
    gen_s = time.perf_counter() - t0
    s = rg.Solver(S.m, S.n, S.row_ptr, S.col_idx, S.vals)
    default = (s.info().lanes_per_row, s.info().lanes_per_col)
    lr, lc, us_r, us_c = rg.rgdbek_tune_spmv(s.handle, reps=10)
    xv = torch.randn(S.n, dtype=torch.float64, device=dev)
    zv = torch.randn(S.m, dtype=torch.float64, device=dev)
    y = torch.empty(S.m, dtype=torch.float64, device=dev)
    g = torch.empty(S.n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    out = {"workload": f"sparse_ls_{S.m}x{S.n}_k{w['k']} (seed {w['seed']})", "nnz": S.nnz,
           "generate_s": gen_s, "default_lanes": {"row": default[0], "col": default[1]},
           "tuned_lanes": {"row": lr, "col": lc},
           "tuner_us": {"csr": {str(k): round(v, 2) for k, v in us_r.items()},
                        "csc": {str(k): round(v, 2) for k, v in us_c.items()}}}
    cases = {"csr_Ax": (lambda: rg.rgdbek_spmv(s.handle, xv, y),
                        12 * S.nnz + 8 * (S.m + 1) + 8 * S.n + 8 * S.m),
             "csc_ATz": (lambda: rg.rgdbek_spmv_t(s.handle, zv, g),
                         12 * S.nnz + 8 * (S.n + 1) + 8 * S.m + 8 * S.n)}
    # the FP32 form's passes: float values and vectors, the same index arrays
    xf, zf = xv.float(), zv.float()
    yf = torch.empty(S.m, dtype=torch.float32, device=dev)
    gf = torch.empty(S.n, dtype=torch.float32, device=dev)
    cases["csr_Ax_f32"] = (lambda: rg.rgdbek_spmv_f32(s.handle, 0, xf, yf),
                           8 * S.nnz + 8 * (S.m + 1) + 4 * S.n + 4 * S.m)
    cases["csc_ATz_f32"] = (lambda: rg.rgdbek_spmv_f32(s.handle, 1, zf, gf),
                            8 * S.nnz + 8 * (S.n + 1) + 4 * S.m + 4 * S.n)
    for name, (fn, nbytes) in cases.items():
        fn()
        ts = []
        for i in range(10):
            a, bb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.fill_(float(i))
            torch.cuda._sleep(400000)
            a.record(stream)
            fn()
            bb.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(bb) / 1e3)
        t = statistics.median(ts)
        gbs = nbytes / t / 1e9
        out[name] = {"us": t * 1e6, "algorithmic_bytes": nbytes, "GB/s": gbs, "frac": gbs / peak,
                     "flop_tflops": 2 * S.nnz / t / 1e12}
        if not name.endswith("_f32"):
            out[name]["fp64_frac_of_nominal"] = 2 * S.nnz / t / 1e12 / FP64_PEAK_TFLOPS
    s.close()
    del S
    return out


def adaptive_inner(rg, S, opts, w, max_iter, b, x_ref, flush, stream, args, c=0.1):
    """Time the solve with inner_adapt = c (inner tolerance
    max(1e-10, min(0.1, c * r_k))) under the same L2 flush, and compare its
    solution with the fixed-tolerance one left in x_ref."""
    import torch
    s = rg.Solver(S.m, S.n, S.row_ptr, S.col_idx, S.vals, inner_adapt=c, **opts)
    x = torch.empty_like(x_ref)
    st = rg.rgdbek_solve(s.handle, b, x, w["tol"], max_iter, 77)
    torch.cuda.synchronize()
    ms, stats = [], []
    for i in range(max(1, min(args.steps, 3))):
        flush.fill_(float(i))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stats.append(rg.rgdbek_solve(s.handle, b, x, w["tol"], max_iter, i))
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    s.close()
    its = sum(t.iters for t in stats)
    st = stats[0]
    return {"inner_adapt": c, "value": its / (sum(ms) / 1e3), "unit": UNIT,
            "time_to_tol_s": statistics.median(ms) / 1e3,
            "iters_per_solve": [t.iters for t in stats],
            "lsqr_steps_per_solve": [t.inner_u + t.inner_j for t in stats],
            "status": [t.status for t in stats],
            "rel_diff_to_fixed_tol_x": float(torch.linalg.norm(x - x_ref) /
                                             torch.linalg.norm(x_ref)),
            "final_normal_res": st.normal_res}


def fp32_inner(rg, S, opts, w, max_iter, b, x_ref, flush, stream, args):
    """The benchmark solve with precision = FP32_INNER: Algorithm 1 in FP32
    (float A values, vectors, weights, LSQR with Kahan dots) inside FP64
    iterative refinement, to the same FP64 normal-equation residual, L2
    flushed before each timed solve."""
    import torch
    s = rg.Solver(S.m, S.n, S.row_ptr, S.col_idx, S.vals, precision=rg.PRECISION_FP32_INNER,
                  **opts)
    x = torch.empty_like(x_ref)
    rg.rgdbek_solve(s.handle, b, x, w["tol"], max_iter, 77)
    torch.cuda.synchronize()
    ms, stats = [], []
    for i in range(max(1, min(args.steps, 3))):
        flush.fill_(float(i))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stats.append(rg.rgdbek_solve(s.handle, b, x, w["tol"], max_iter, i))
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    s.close()
    st = stats[-1]
    return {"time_to_tol_s": statistics.median(ms) / 1e3,
            "iters_per_solve": [t.iters for t in stats],
            "refinements_per_solve": [t.refinements for t in stats],
            "lsqr_steps_per_solve": [t.inner_u + t.inner_j for t in stats],
            "status": [t.status for t in stats],
            "final_normal_res": st.normal_res,
            "phase_ms": {k: round(v, 3) for k, v in st.as_dict()["phase_ms"].items()},
            "us_per_grid_phase": 1e6 * statistics.median(ms) / 1e3 / max(
                1, 14 * st.iters + 2 * (st.inner_u + st.inner_j) + 4 * st.refinements),
            "rel_diff_to_fp64_x": float(torch.linalg.norm(x - x_ref) / torch.linalg.norm(x_ref))}


def eta_tuning(rg, S, opts, w, max_iter, b, flush, stream, probe_iters=20):
    """rgdbek_tune_eta over its default candidates (probe_iters iterations
    each), then one L2-flushed solve to the tolerance at every candidate, so
    the tuner's choice can be checked against the measured best."""
    import torch
    o = dict(opts)
    o.pop("eta_col", None)
    o.pop("eta_row", None)
    s = rg.Solver(S.m, S.n, S.row_ptr, S.col_idx, S.vals, eta_col=w["eta"], eta_row=w["eta"], **o)
    x = torch.empty(S.n, dtype=torch.float64, device=b.device)
    best, scores = s.tune_eta(b, probe_iters=probe_iters, seed=5)
    per = {}
    for c in rg.ETA_CANDIDATES:
        s.set_options(eta_col=c, eta_row=c)
        flush.fill_(c)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = rg.rgdbek_solve(s.handle, b, x, w["tol"], max_iter, 3, raise_on_error=False)
        e1.record(stream)
        torch.cuda.synchronize()
        per[str(c)] = {"time_to_tol_s": e0.elapsed_time(e1) / 1e3, "iters": st.iters,
                       "status": st.status, "tuner_score": scores[c]}
    s.close()
    fastest = min(per, key=lambda k: per[k]["time_to_tol_s"] if per[k]["status"] == 0 else 1e30)
    return {"probe_iters": probe_iters, "tuned_eta": best, "fastest_eta": float(fastest),
            "by_eta": per}


def end_to_end(rg, S, opts, w, max_iter, args):
    import torch
    rp = torch.from_numpy(S.row_ptr).pin_memory()
    ci = torch.from_numpy(S.col_idx).pin_memory()
    av = torch.from_numpy(S.vals).pin_memory()
    b = torch.from_numpy(S.b).pin_memory()
    x = torch.empty(S.n, dtype=torch.float64).pin_memory()
    o = rg.default_options(**opts)

    def step(seed):
        h = rg._ptr()
        st = rg._lib.rgdbek_create(rg.ctypes.byref(h), S.m, S.n, S.nnz, rp.data_ptr(),
                                   ci.data_ptr(), av.data_ptr(), 0, rg.ctypes.byref(o),
                                   torch.cuda.current_stream().cuda_stream)
        rg._check(st, "rgdbek_create")
        res = rg.rgdbek_solve_host(h.value, b, x, w["tol"], max_iter, seed)
        rg.rgdbek_destroy(h.value)
        return res

    nsteps = max(1, min(args.steps, 3))
    step(99)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    its = 0
    for i in range(nsteps):
        its += step(i).iters
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    h2d = 8 * (S.m + 1) + 12 * S.nnz + 8 * S.m
    d2h = 8 * S.n + 256
    return {"value": its / dt, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "steps": nsteps,
            "what": "rgdbek_create from pinned host CSR + rgdbek_solve_host + destroy per step"}


def _setup_gpu():
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "_rgdbek_build", os.path.join(ROOT, "paper_2509_19267_gb300", "build.py"))
    bmod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bmod)
    bmod.build()
    import paper_2509_19267_gb300 as rg
    return torch, rg


def _timed(torch, fn, steps):
    stream = torch.cuda.current_stream()
    ms, outs = [], []
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        outs.append(fn())
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return ms, outs


def run_batched_deblur(args):
    """Many uneven systems in one persistent launch, against one solve after
    another; a fixed budget of outer iterations per system."""
    torch, rg = _setup_gpu()
    budget = args.budget or 10
    t0 = time.perf_counter()
    S = workloads.blur_batch(args.batch_count, 64, 512, seed=3)
    gen_s = time.perf_counter() - t0
    opts = dict(eta_col=0.1, eta_row=0.1, stop_rule=rg.STOP_REL_RES)
    if args.inner_max:
        opts["inner_max"] = args.inner_max
    if args.fp32:
        opts["precision"] = rg.PRECISION_FP32_INNER
    hs = [rg.Solver(s.m, s.n, s.row_ptr, s.col_idx, s.vals, **opts) for s in S]
    H = [h.handle for h in hs]
    bs = [torch.from_numpy(s.b).cuda() for s in S]
    xs = [torch.empty(s.n, dtype=torch.float64, device="cuda") for s in S]
    tols = [1e-8] * len(S)
    team, tuned_block, tune_ms, shape_ms = rg.rgdbek_tune_batched(H, bs, xs, tols, probe_iters=2)
    for _ in range(args.warmup):
        rg.rgdbek_solve_batched(H, bs, xs, tols, budget, seed=0)
    clocks = ClockSampler(0)
    clocks.start()
    ms, outs = _timed(torch, lambda: rg.rgdbek_solve_batched(H, bs, xs, tols, budget, seed=0),
                      args.steps)
    clk = clocks.stop()
    iters = sum(st.iters for st in outs[0][1])
    value = iters * args.steps / (sum(ms) / 1e3)

    def sequential():
        its = 0
        for h, b, x in zip(hs, bs, xs):
            its += rg.rgdbek_solve(h.handle, b, x, 1e-8, budget, 0).iters
        return its

    sequential()
    ms_seq, outs_seq = _timed(torch, sequential, 1)
    seq_value = outs_seq[0] / (ms_seq[0] / 1e3)
    rel = [st.rel_res for st in outs[0][1]]
    # roofline of the batched launch: the algorithmic bytes of every system's
    # solve (from its own counters) over the launch's CUDA-event time
    peak, peak_kind = measured_peaks()
    sts = outs[0][1]
    alg = sum(algorithmic_bytes(st, s.m, s.n, s.nnz) for st, s in zip(sts, S))
    t_launch = statistics.median(ms) / 1e3
    inner_max = opts.get("inner_max", 200)
    row_steps = [st.inner_j / max(st.iters, 1) for st in sts]
    line = {"metric": f"batched RGDBEK system-iterations/s ({len(S)} deblur systems, "
                      f"{budget}-iteration budget each)",
            "value": value, "unit": "system-iters/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.mean(ms),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"blur_batch_{len(S)}_sides64-512", "systems": len(S),
                       "unknowns": int(sum(s.n for s in S)), "nnz": int(sum(s.nnz for s in S)),
                       "eta": 0.1, "budget": budget, "team": team,
                       "teams": hs[0].info().grid // team,
                       "l2": "inputs larger than L2 (25 GB of CSR)"},
            "tuner_ms": {str(k): v for k, v in tune_ms.items()},
            "tuner_shape_ms": {str(k): v for k, v in shape_ms.items()},
            "block": tuned_block or "automatic",
            "sequential": {"value": seq_value, "unit": "system-iters/s",
                           "ms": ms_seq[0], "what": "rgdbek_solve per system, whole GPU each"},
            "speedup_vs_sequential": value / seq_value,
            "rel_res_after_budget": {"min": min(rel), "median": statistics.median(rel),
                                     "max": max(rel)},
            "roofline": {"bound": "hbm", "achieved": alg / t_launch / 1e9, "peak": peak,
                         "unit": "GB/s", "frac": alg / t_launch / 1e9 / peak, "traffic": None,
                         "kernel": "batched_solve_kernel (one launch per step)",
                         "peak_source": peak_kind, "algorithmic_bytes_per_launch": alg},
            "inner_max": inner_max,
            "row_lsqr_steps_per_iteration": {"min": min(row_steps),
                                             "median": statistics.median(row_steps),
                                             "max": max(row_steps)},
            "col_lsqr_steps_per_iteration": statistics.median(
                [st.inner_u / max(st.iters, 1) for st in sts]),
            "precision": "fp32 inner / fp64 refinement" if args.fp32 else "fp64",
            "generate_s": gen_s, "gpu_launches": args.steps * 4, "clocks": clk}
    print(json.dumps(line), flush=True)
    for h in hs:
        h.close()


def run_poisson_mixed(args):
    """FP32 inner products against FP64 on the P1 Poisson system, fixed budget."""
    torch, rg = _setup_gpu()
    budget = args.budget or 500
    S = workloads.poisson_p1(1024, seed=2)
    b = torch.from_numpy(S.b).cuda()
    res = {}
    xs = {}
    for name, prec in (("fp64", rg.PRECISION_FP64), ("fp32_inner", rg.PRECISION_FP32_INNER)):
        h = rg.Solver(S.m, S.n, S.row_ptr, S.col_idx, S.vals, eta_col=0.1, eta_row=0.1,
                      stop_rule=rg.STOP_REL_RES, precision=prec, inner_tol=1e-6)
        x = torch.empty(S.n, dtype=torch.float64, device="cuda")
        for _ in range(args.warmup):
            rg.rgdbek_solve(h.handle, b, x, 1e-8, min(budget, 20), 0)
        ms, outs = _timed(torch, lambda: rg.rgdbek_solve(h.handle, b, x, 1e-8, budget, 0),
                          args.steps)
        st = outs[-1]
        res[name] = {"iters_per_s": st.iters * args.steps / (sum(ms) / 1e3),
                     "ms_per_solve": statistics.mean(ms), "iters": st.iters,
                     "rel_res": st.rel_res,
                     "lsqr_steps_per_iter": (st.inner_u + st.inner_j) / max(st.iters, 1)}
        xs[name] = x.clone()
        h.close()
    diff = float(torch.linalg.norm(xs["fp32_inner"] - xs["fp64"]) / torch.linalg.norm(xs["fp64"]))
    xstar = torch.from_numpy(S.x_true).cuda()
    line = {"metric": f"P1 Poisson 1024x1024 outer iterations/s, FP32 inner products "
                      f"({budget}-iteration budget)",
            "value": res["fp32_inner"]["iters_per_s"], "unit": "iters/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": res["fp32_inner"]["ms_per_solve"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 inner / f64 outer",
            "data": "synthetic",
            "config": {"workload": "poisson_p1_1024x1024", "unknowns": S.n, "nnz": S.nnz,
                       "eta": 0.1, "budget": budget, "inner_tol": 1e-6,
                       "l2": "inputs larger than L2 after the solver's workspace"},
            "fp64": res["fp64"], "fp32_inner": res["fp32_inner"],
            "speedup_vs_fp64": res["fp32_inner"]["iters_per_s"] / res["fp64"]["iters_per_s"],
            "rel_diff_x_fp32_vs_fp64": diff,
            "rel_err_vs_x_star": {k: float(torch.linalg.norm(v - xstar) / torch.linalg.norm(xstar))
                                  for k, v in xs.items()},
            "gpu_launches": 2 * args.steps}
    print(json.dumps(line), flush=True)


def run_deblur_adjoint(args):
    """Forward solve and implicit adjoint on the regularised 256 x 256 deblur."""
    torch, rg = _setup_gpu()
    S = workloads.deblur_regularised(256)
    b = torch.from_numpy(S.b).cuda()
    xt = torch.from_numpy(S.x_true).cuda()
    out = {}
    for name, prec in (("fp64", rg.PRECISION_FP64), ("fp32_inner", rg.PRECISION_FP32_INNER)):
        h = rg.Solver(S.m, S.n, S.row_ptr, S.col_idx, S.vals, eta_col=0.1, eta_row=0.1,
                      stop_rule=rg.STOP_NORMAL, precision=prec)
        fwd = h.solve(b, tol=1e-10, max_iter=200000, seed=0)
        x = fwd.x
        g = 2.0 * (x - xt)
        steps = max(1, min(args.steps, 2))
        ms, outs = _timed(torch, lambda: h.backward(b, x, g, tol=1e-10, max_iter=200000,
                                                    seed=1, nnz=S.nnz), steps)
        gb, gv, status, st = outs[-1]
        gx = float(torch.dot(g, x))
        out[name] = {"backward_s": statistics.mean(ms) / 1e3, "status": status,
                     "solve_iters": [st[0].iters, st[1].iters],
                     "forward_iters": fwd.stats.iters,
                     "identity_db": abs(float(torch.dot(gb, b)) - gx) / abs(gx),
                     "identity_dA": abs(float(torch.dot(gv, torch.from_numpy(S.vals).cuda())) + gx)
                     / abs(gx)}
        h.close()
    line = {"metric": "implicit adjoint of the regularised 256x256 deblur: backward passes/s",
            "value": 1.0 / out["fp64"]["backward_s"], "unit": "backward/s", "n_gpus": 1,
            "steps": args.steps, "warmup": 0, "ms_per_step": 1e3 * out["fp64"]["backward_s"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "deblur_regularised_256x256_lam0.05", "m": S.m, "n": S.n,
                       "nnz": S.nnz, "eta": 0.1, "tol": 1e-10,
                       "loss": "||x - x_true||^2"},
            "fp64": out["fp64"], "fp32_inner": out["fp32_inner"],
            "gpu_launches": 6 * args.steps}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched_deblur":
        run_batched_deblur(args)
    elif args.workload == "poisson_mixed":
        run_poisson_mixed(args)
    elif args.workload == "deblur_adjoint":
        run_deblur_adjoint(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
