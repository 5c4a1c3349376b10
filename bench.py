"""Benchmark: ms per 200K-point Faster Mean-shift clustering on GB300.

One step = one fms_cluster call (Seed Selection, mean-shift updates under
Early Stopping, prune, seed doubling, FP64-accumulated refinement, labels) on
the paper-scale 3-D workload: n = 200,000 points, 20 Dirichlet-sized blobs plus
2% uniform noise, h = 5 (synthetic stand-in for the paper's 200K-point Table I
case).  Inputs are resident in HBM when the timed region starts; L2 is flushed
(256 MB write) between timed steps, outside the per-step CUDA events.

Extra measurements on the same line:
  roofline      the dominant kernel (the grid round): seed-point evaluations
                per second from CUDA events around each launch, against the
                FP32 pipe bound of the exact-difference evaluation the kernel
                runs (3d+1 FP32 ops per eval; frac_2d2: the same against the
                minimal 2d+2 count); frac_measured divides by the FFMA rate the
                library measures on this GPU in this run (fms_probe_pipe_rates).
  accuracy      the timed clustering against the FP64 oracle's: largest mode
                error / h, labels that differ away from near-ties, points
                whose oracle margin is below 1e-2 h, mode counts and order.
  all_seeds     the plain all-seeds GPU path (Alg. 1) on the same points: its
                time, the speedup of the faster path over it, and how its modes
                and labels compare with the faster path's on the blobs.
  e2e           the same clustering through the C ABI with host buffers: the
                pinned host -> device copy of the points and the device -> host
                copy of labels and modes are inside the timed region.
  cpu_baseline  the FP64 oracle on the host cores (rank 0, N = 1 only).
  clocks        nvidia-smi samples taken during the timed region.

--impl reference times the FP64 oracle (the reference arm of this project) on
the same workload and prints the same line with "impl": "reference".
Multi-GPU (torchrun): independent replicas, one point set per rank, no
data-path collective ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "ms per 200K-point clustering"
N_POINTS, DIM = 200_000, 3
SM_COUNT = 152
FP32_LANES_PER_SM = 128


def workload_desc():
    return {"workload": "paper_3d: n=200000 points in 3-D, 20 Gaussian blobs (centres U[0,200]^3, "
                        "sigma U[1,3], Dirichlet(2) sizes) + 2% uniform noise, h=5, tol=1e-3*h; "
                        "Seed Selection (N0=128, L=8) + Early Stopping (gamma=0.95), FP64 refine",
            "n": N_POINTS, "d": DIM, "h": 5.0,
            "l2": "flushed between timed steps (256 MB write outside the step events)"}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_input(rank):
    """Rank r clusters its own seeded point set (independent problems, no data-path collective)."""
    import fms_inputs as fi
    return fi.paper_3d(seed=rank)


def reduce_max(x, pg, device):
    """Max over the ranks of a float (the value itself without a process group)."""
    if pg is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_ms_per_clustering(t_total_ms, steps, world, pg, device):
    """Whole-job time per clustering: the slowest rank's timed total over the clusterings that
    all ranks ran together (each rank runs `steps`); also returns ms per step (max over ranks)."""
    t = reduce_max(t_total_ms, pg, device)
    return t / (steps * world), t / steps


def reference_runs_on(rank):
    """The reference (oracle) arm runs on rank 0 only; other ranks exit without work."""
    return rank == 0


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(parts)
            except Exception:
                pass
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i]
                          and "Not" not in r[5 + i]})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path))
    except Exception:
        return {}


# Source files whose contents fix each profiled kernel's code: a stored DRAM
# traffic figure counts only while their digest matches the one it was taken at.
KERNEL_SOURCES = {
    "ms_grid_round": ["paper_2112_13891_gb300/csrc/k_grid.cu",
                      "paper_2112_13891_gb300/csrc/fms_internal.cuh"],
    "ms_step": ["paper_2112_13891_gb300/csrc/k_step.cu",
                "paper_2112_13891_gb300/csrc/fms_step_body.cuh",
                "paper_2112_13891_gb300/csrc/fms_internal.cuh"],
    "ms_step_tc": ["paper_2112_13891_gb300/csrc/k_step_tc.cu",
                   "paper_2112_13891_gb300/csrc/fms_tc.cuh",
                   "paper_2112_13891_gb300/csrc/fms_internal.cuh"],
}


def source_digest(kname):
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES[kname]:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(rel.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


def stored_traffic(kname):
    """DRAM bytes per launch from profiles/<kernel>_traffic.json, or None when
    the file is missing or the kernel's sources changed since the capture."""
    tfile = os.path.join(ROOT, "profiles", f"{kname}_traffic.json")
    if not os.path.exists(tfile):
        return None
    try:
        rec = json.load(open(tfile))
    except (OSError, ValueError):
        return None
    if rec.get("source_digest") != source_digest(kname):
        return None
    return rec.get("bytes_per_launch")


def run_oracle_sample(w, seconds=12.0):
    """Time the FP64 oracle's full clustering of the workload on the host cores;
    also returns the oracle's result (for the accuracy record)."""
    import oracle as orc
    t0 = time.perf_counter()
    runs = 0
    while True:
        ref = orc.cluster(w.X, w.h, w.tol, w.max_iter, gamma=0.95, rng_seed=0)
        runs += 1
        el = time.perf_counter() - t0
        if el >= seconds or runs >= 20:
            break
    return el / runs * 1e3, runs, ref


def accuracy_vs_oracle(modes, labels, ref, h, mode_tol=1e-3, margin_tol=1e-2, score_rtol=1e-4):
    """GPU clustering against the FP64 oracle: modes matched one-to-one
    (Hungarian assignment on distances), labels compared after that mapping
    away from near-ties (oracle margin >= margin_tol h), the canonical order
    checked up to near-equal oracle scores."""
    from scipy.optimize import linear_sum_assignment
    g = np.asarray(modes, dtype=np.float64)
    r = np.asarray(ref.modes, dtype=np.float64)
    out = {"n_modes": int(g.shape[0]), "n_modes_oracle": int(r.shape[0])}
    if g.shape != r.shape:
        out["mode_count_equal"] = False
        return out
    D = np.sqrt(((g[:, None, :] - r[None, :, :]) ** 2).sum(-1))
    gi, ri = linear_sum_assignment(D)
    perm = np.empty(g.shape[0], dtype=np.int64)
    perm[gi] = ri
    err = float(D[gi, ri].max()) if len(gi) else 0.0
    lab = np.asarray(labels).astype(np.int64)
    mapped = np.where(lab >= 0, perm[np.clip(lab, 0, None)], -1)
    keep = ref.margins >= margin_tol * h
    s = np.asarray(ref.scores, dtype=np.float64)[perm]
    i, j = np.triu_indices(perm.shape[0], k=1)
    viol = int(((perm[i] > perm[j]) &
                (np.abs(s[i] - s[j]) > score_rtol * np.maximum(np.abs(s[i]), np.abs(s[j])))).sum())
    out.update({"mode_count_equal": True, "max_mode_err_over_h": err / h,
                "modes_within_1e-3h": bool(err <= mode_tol * h),
                "label_mismatch": int((mapped[keep] != ref.labels[keep]).sum()),
                "low_margin_points": int((~keep).sum()), "order_violations": viol,
                "n_seeds_oracle": int(ref.n_seeds)})
    return out


def oracle_one_core_ms(seconds):
    """The same oracle sample on one host core: a child process started with
    OMP_NUM_THREADS=1 (OpenMP fixes its thread count when the library loads)."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample-only",
                        str(seconds)], env=env, capture_output=True, text=True,
                       timeout=max(120.0, 20 * seconds))
    if r.returncode != 0:
        return None, 0
    out = json.loads(r.stdout.strip().splitlines()[-1])
    return out["ms"], out["runs"]


def oracle_threads():
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v else (os.cpu_count() or 1)


def bench_reference(args):
    rank, world, _ = dist_env()
    if not reference_runs_on(rank):
        return
    w = make_input(0)
    import oracle as orc
    for _ in range(args.warmup):
        orc.cluster(w.X, w.h, w.tol, w.max_iter, gamma=0.95, rng_seed=0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        orc.cluster(w.X, w.h, w.tol, w.max_iter, gamma=0.95, rng_seed=0)
    ms = (time.perf_counter() - t0) / args.steps * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": ms, "unit": "ms",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_desc(),
            "cpu_baseline": {"value": ms, "unit": "ms", "cores": oracle_threads(), "kind": "oracle",
                             "sample": f"full FP64 oracle clustering of the workload, {args.steps} runs"},
            "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def bench_fms(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    import paper_2112_13891_gb300 as fms

    w = make_input(rank)
    X = torch.from_numpy(w.X).to(dev)
    n, d = X.shape
    ws = fms.Workspace(fms.workspace_size(n, d), dev)
    modes = torch.empty((n, d), dtype=torch.float32, device=dev)
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    margins = torch.empty(n, dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step(profile=False):
        return fms.cluster(X, w.h, w.tol, w.max_iter, gamma=0.95, rng_seed=0, workspace=ws,
                           out=(modes, labels, margins), profile=profile)

    def barrier():
        torch.cuda.synchronize()
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    for _ in range(max(args.warmup, 3)):
        r = step()
    st = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(torch.cuda.current_device())
    barrier()
    clocks.start()
    time.sleep(0.5)          # let nvidia-smi start sampling before the timed steps
    t_wall = time.perf_counter()
    launches = 0
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(st)
        r = step()
        ev[i][1].record(st)
        launches += r.stats["kernel_launches"] + 0
    barrier()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    value, ms_per_step = job_ms_per_clustering(float(sum(step_ms)), args.steps, world, pg, dev)

    # --- roofline of the dominant kernel: CUDA events around each launch (profile mode) ---
    prof = {"step_ms": 0.0, "step_ev": 0, "step_n": 0, "round_ms": 0.0, "round_ev": 0,
            "round_n": 0, "phase": [0.0, 0.0, 0.0, 0.0]}
    barrier()
    for i in range(args.steps):
        flush.zero_()
        rp = step(profile=True).stats
        prof["step_ms"] += rp["step_kernel_ms"]
        prof["step_ev"] += rp["step_evals"]
        prof["step_n"] += rp["step_launches"]
        prof["round_ms"] += rp["round_kernel_ms"]
        prof["round_ev"] += rp["round_evals"]
        prof["round_n"] += rp["round_launches"]
        prof["phase"] = [a + b for a, b in zip(prof["phase"], rp["phase_ms"])]
    barrier()
    if prof["round_ms"] >= prof["step_ms"] and prof["round_n"] > 0:
        kname, kms, kev, kn = "ms_grid_round", prof["round_ms"], prof["round_ev"], prof["round_n"]
    else:
        kname, kms, kev, kn = "ms_step", prof["step_ms"], prof["step_ev"], prof["step_n"]
    avg_launch_ms = kms / max(kn, 1)
    evals_per_launch = kev / max(kn, 1)
    achieved = evals_per_launch / (avg_launch_ms * 1e-3) / 1e9          # Geval/s
    ops_per_eval = 3 * d + 1          # the exact-difference evaluation the kernels run
    ops_minimal = 2 * d + 2           # the minimal (expanded) formulation
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak = SM_COUNT * FP32_LANES_PER_SM * sm_max * 1e6 / ops_per_eval / 1e9
    peak_min = SM_COUNT * FP32_LANES_PER_SM * sm_max * 1e6 / ops_minimal / 1e9
    try:
        rates = fms.probe_pipe_rates()
    except Exception:
        rates = None
    peak_meas = None
    if rates and rates["ffma_ops_per_clk_sm"] > 0:
        # the same bound from the FFMA rate measured here, at the maximum clock
        peak_meas = SM_COUNT * rates["ffma_ops_per_clk_sm"] * sm_max * 1e6 / ops_per_eval / 1e9
    traffic = stored_traffic(kname)
    phases = {k: v / args.steps for k, v in zip(("rounds", "prunes", "refine", "labels"),
                                               prof["phase"])}

    # --- end to end through the C ABI with host buffers (fms_cluster_host:
    # the points uploaded, the labels and modes copied back, in one call; the
    # buffers are page-locked, so the call's kernels read the points and write
    # the labels over the CPU-GPU link themselves, inside the timed region) ---
    cap_h = 256
    Xh = torch.from_numpy(w.X).pin_memory()
    lab_h = torch.empty(n, dtype=torch.int32).pin_memory()
    modes_h = torch.empty((cap_h, d), dtype=torch.float32).pin_memory()
    ws_h = fms.Workspace(int(fms._lib.fms_cluster_host_workspace_size(
        n, d, cap_h, ctypes.byref(fms.make_options(gamma=0.95, rng_seed=0)))),
        X.device)
    run_h = lambda: fms.cluster_host(Xh, w.h, w.tol, w.max_iter, gamma=0.95, rng_seed=0,
                                     workspace=ws_h, out=(modes_h, lab_h, None))
    for _ in range(max(3, args.warmup)):
        run_h()
    barrier()
    e2e_ms = []
    for i in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        run_h()
        b.record(st)
        b.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    # labels, the modes buffer and the 1 KB control region the call reads back
    d2h_bytes = n * 4 + cap_h * d * 4 + 1024
    e2e = reduce_max(float(np.mean(e2e_ms)), pg, dev) / world

    # --- the plain all-seeds path (Alg. 1) on the same points: time and agreement ---
    all_seeds = None
    if rank == 0 and world == 1 and not args.no_all_seeds:
        fast_modes = r.modes.cpu().numpy().astype(np.float64)
        fast_labels = labels.cpu().numpy().astype(np.int64)
        fast_margins = margins.cpu().numpy()
        ws_a = fms.Workspace(fms.workspace_size(n, d), dev)
        run_a = lambda: fms.cluster(X, w.h, w.tol, w.max_iter, all_seeds=True, workspace=ws_a)
        ra = run_a()
        t_a, _ = _events_ms(run_a, 2, flush=flush)
        A = ra.modes.cpu().numpy().astype(np.float64)
        la = ra.labels.cpu().numpy().astype(np.int64)
        # every faster-path mode against its nearest all-seeds mode
        DA = np.sqrt(((fast_modes[:, None, :] - A[None, :, :]) ** 2).sum(-1))
        near = DA.argmin(axis=1)
        near_d = DA[np.arange(DA.shape[0]), near]
        # labels: points the all-seeds path gives to a mode that matches a
        # faster-path mode, compared away from the faster path's near-ties
        a2f = np.full(A.shape[0], -1, dtype=np.int64)
        ok_m = near_d <= 1e-3 * w.h
        a2f[near[ok_m]] = np.nonzero(ok_m)[0]
        mapped = a2f[la]
        on_blobs = mapped >= 0
        firm = fast_margins >= 1e-2 * w.h
        cmp = on_blobs & firm
        all_seeds = {"ms": t_a, "speedup_of_faster_path": t_a / value,
                     "n_modes": int(A.shape[0]), "n_modes_faster_path": int(fast_modes.shape[0]),
                     "max_dist_faster_mode_to_all_seeds_mode_over_h": float(near_d.max() / w.h),
                     "faster_modes_matched_within_1e-3h": int(ok_m.sum()),
                     "points_on_matched_modes": int(on_blobs.sum()),
                     "label_agreement_on_matched_modes": float((mapped[cmp] == fast_labels[cmp]).mean())
                     if cmp.any() else None,
                     "label_mismatch_on_matched_modes": int((mapped[cmp] != fast_labels[cmp]).sum()),
                     "evals": int(ra.stats["evals"])}
        del ws_a

    cpu = None
    accuracy = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ms_cpu, runs, ref = run_oracle_sample(w, seconds=args.cpu_seconds)
        accuracy = accuracy_vs_oracle(r.modes.cpu().numpy(), labels.cpu().numpy(), ref, w.h)
        cpu = {"value": ms_cpu, "unit": "ms", "cores": oracle_threads(), "kind": "oracle",
               "sample": f"full FP64 oracle clustering of the same 200K-point workload, "
                         f"{runs} run(s), OpenMP over seeds"}
        ms_one, runs_one = oracle_one_core_ms(args.cpu_seconds)
        if ms_one is not None:
            cpu["value_1_core"] = ms_one
            cpu["sample_1_core"] = f"the same clustering on one host core, {runs_one} run(s)"
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "ms", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic", "config": dict(workload_desc(), parallelism=f"replicas{world}"),
                "roofline": {"bound": "alu", "kernel": kname, "achieved": achieved,
                             "peak": peak, "unit": "Geval/s", "frac": achieved / peak,
                             "traffic": traffic,
                             "peak_basis": f"FP32 pipe {FP32_LANES_PER_SM} lanes/clk/SM x {SM_COUNT} SMs x "
                                           f"{sm_max:.0f} MHz / {ops_per_eval} FP32 ops per eval (3d+1, "
                                           f"the exact-difference form the kernel runs)",
                             "frac_2d2": achieved / peak_min,
                             "peak_2d2": peak_min,
                             "frac_measured": achieved / peak_meas if peak_meas else None,
                             "peak_measured": peak_meas,
                             "pipe_rates_per_clk_sm": rates,
                             "avg_launch_us": avg_launch_ms * 1e3,
                             "evals_per_launch": evals_per_launch, "launches": kn,
                             "share_of_step": kms / max(sum(prof["phase"]), 1e-9)},
                "phase_ms": phases,
                "evals_per_s": r.stats["evals"] / (ms_per_step * 1e-3),
                "e2e": {"value": e2e, "unit": "ms", "h2d_bytes_per_step": n * d * 4,
                        "d2h_bytes_per_step": d2h_bytes},
                "cpu_baseline": cpu, "accuracy": accuracy, "all_seeds": all_seeds,
                "clocks": clk, "gpu_launches": launches,
                "wall_s_timed": wall,
                "stats": {k: r.stats[k] for k in ("iterations", "rounds", "n_seeds_final",
                                                   "n_modes", "refine_iterations", "evals",
                                                   "score_evals", "kernel_launches")}}
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


def kernel_probe(m, reps=3):
    """One ms_step-only case: m seeds (the first m points) against all 200K points."""
    import torch
    import paper_2112_13891_gb300 as fms
    w = make_input(0)
    X = torch.from_numpy(w.X).cuda()
    Y = X[:m].clone()
    ws = fms.Workspace(fms._lib.fms_step_workspace_size(X.shape[0], X.shape[1], m), X.device)
    for _ in range(reps):
        out = fms.mean_shift_step(X, Y, w.h, workspace=ws)
    torch.cuda.synchronize()
    print(json.dumps({"kernel_probe": m, "first": out[0].tolist()}))


def _events_ms(fn, reps, flush=None):
    import torch
    out = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        out.append(a.elapsed_time(b))
    return float(np.median(out)), out


def bench_extra(args):
    """Measurements of the other hot-path rows (one JSON line each; not the headline)."""
    import torch
    import fms_inputs as fi
    import paper_2112_13891_gb300 as fms
    torch.cuda.set_device(0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    line = {"workload": args.workload, "data": "synthetic"}
    if args.workload == "all_seeds_3d":
        w = fi.paper_3d()
        X = torch.from_numpy(w.X).cuda()
        ws = fms.Workspace(fms.workspace_size(X.shape[0], 3, all_seeds=True), X.device)
        run = lambda: fms.cluster(X, w.h, w.tol, w.max_iter, all_seeds=True, workspace=ws)
        r = run()
        ms, _ = _events_ms(run, max(2, args.steps // 50), flush)
        rp = fms.cluster(X, w.h, w.tol, w.max_iter, all_seeds=True, workspace=ws, profile=True)
        st = rp.stats
        fast = fms.cluster(X, w.h, w.tol, w.max_iter, workspace=fms.Workspace(
            fms.workspace_size(X.shape[0], 3), X.device))
        fms_ms, _ = _events_ms(lambda: fms.cluster(X, w.h, w.tol, w.max_iter), 20, flush)
        line.update({"metric": "ms per 200K-point clustering, every point a seed (Alg. 1)",
                     "value": ms, "unit": "ms", "n_modes": r.stats["n_modes"],
                     "evals": r.stats["evals"], "evals_per_s": r.stats["evals"] / (ms * 1e-3),
                     "step_kernel": {"launches": st["step_launches"], "ms": st["step_kernel_ms"],
                                     "evals_per_s": st["step_evals"] / max(st["step_kernel_ms"], 1e-9) * 1e3},
                     "faster_path_ms": fms_ms, "speedup_faster_over_all_seeds": ms / fms_ms,
                     "faster_path_modes": fast.stats["n_modes"]})
    elif args.workload == "batched_16d":
        sets = fi.batched_16d()
        X = [torch.from_numpy(w.X).cuda() for w in sets]
        Xc = torch.cat(X)
        offs = np.concatenate([[0], np.cumsum([x.shape[0] for x in X])]).astype(np.int64)
        ws = fms.Workspace(fms._lib.fms_batched_workspace_size(
            offs.ctypes.data_as(ctypes.c_void_p), len(X), 16,
            ctypes.byref(fms.make_options())), Xc.device)
        run = lambda: fms.cluster_batched(Xc, 2.5, 2.5e-3, 300, offsets=offs, max_modes=128,
                                          workspace=ws)
        r = run()   # first call tunes the tiling
        ms, _ = _events_ms(run, 5, flush)
        wss = fms.Workspace(max(fms.workspace_size(x.shape[0], 16) for x in X), Xc.device)
        loop = lambda: [fms.cluster(x, 2.5, 2.5e-3, 300, workspace=wss, max_modes=128) for x in X]
        one = [(o.modes.clone(), o.labels.clone()) for o in loop()]
        ms_loop, _ = _events_ms(loop, 3, flush)
        # equal accuracy: the batched result of every set against its own
        # single-set call (same seeds, same rules)
        same_count, max_diff, agree = 0, 0.0, 0
        for b in range(len(X)):
            mb, lb = r.modes[b], r.labels[int(offs[b]):int(offs[b + 1])]
            if mb.shape == one[b][0].shape:
                same_count += 1
                if mb.numel():
                    max_diff = max(max_diff, (mb - one[b][0]).abs().max().item() / 2.5)
            agree += int((lb == one[b][1]).sum().item())
        line.update({"metric": "ms per batch of 256 point sets (3.2M points, d=16)",
                     "value": ms, "unit": "ms", "per_set_calls_ms": ms_loop,
                     "speedup_batched_over_per_set": ms_loop / ms,
                     "total_points": int(offs[-1]), "evals": r.stats["evals"],
                     "kernel_launches": r.stats["kernel_launches"],
                     "graph": r.stats["graph"], "rounds": r.stats["rounds"],
                     "accuracy_vs_per_set_calls": {
                         "sets_with_equal_mode_count": same_count, "sets": len(X),
                         "max_mode_diff_over_h": max_diff,
                         "label_agreement": agree / float(offs[-1])}})
    elif args.workload == "unrolled_16d":
        w = fi.unrolled_16d()
        X = torch.from_numpy(w.X).cuda()
        G = torch.randn_like(X)
        fwd = lambda: fms.unrolled_forward(X, X, w.h, w.T, w.k_ckpt)
        out, ck = fwd()
        ms_f, _ = _events_ms(fwd, 3)
        bwd = lambda: fms.unrolled_backward(X, ck, X.shape[1], w.h, w.T, w.k_ckpt, G)
        bwd()
        ms_b, _ = _events_ms(bwd, 3)
        B, n, d = X.shape
        pairs = B * n * n * w.T
        line.update({"metric": "ms per forward / backward of 20 unrolled steps (8 x 16384 x 16)",
                     "forward_ms": ms_f, "backward_ms": ms_b, "unit": "ms",
                     "forward_evals_per_s": pairs / (ms_f * 1e-3),
                     "backward_pair_evals_per_s": 3 * pairs / (ms_b * 1e-3)})
    elif args.workload == "embedding_32d":
        w = fi.embedding_32d()
        X = torch.from_numpy(w.X).cuda()
        line.update({"metric": "ms per 65,536-point d=32 clustering", "unit": "ms"})
        for prec in ("tensor", "fp32"):
            ws = fms.Workspace(fms.workspace_size(X.shape[0], 32, precision=prec), X.device)
            run = lambda: fms.cluster(X, w.h, w.tol, w.max_iter, workspace=ws, precision=prec)
            r = run()
            ms, _ = _events_ms(run, max(1, min(10, args.steps)), flush)
            st = fms.cluster(X, w.h, w.tol, w.max_iter, workspace=ws, precision=prec,
                             profile=True).stats
            rec = {"ms": ms, "n_modes": r.stats["n_modes"], "iterations": r.stats["iterations"],
                   "evals": r.stats["evals"], "evals_per_s": r.stats["evals"] / (ms * 1e-3),
                   "fp32_step": {"launches": st["step_launches"], "ms": st["step_kernel_ms"],
                                 "evals": st["step_evals"]},
                   "coarse_step": {"launches": st["coarse_launches"],
                                   "ms": st["coarse_kernel_ms"], "evals": st["coarse_evals"]},
                   "phase_ms": st["phase_ms"]}
            line[prec] = rec
        line["value"] = line["tensor"]["ms"]
        # the same data with every point a seed (Alg. 1): 65,536 seeds keep the
        # tensor-core step at full load; the two precisions are compared with
        # each other (modes matched within 1e-3 h, labels of matched modes)
        if not args.no_all_seeds:
            allr = {}
            for prec in ("tensor", "fp32"):
                ws = fms.Workspace(fms.workspace_size(X.shape[0], 32, precision=prec,
                                                      all_seeds=True), X.device)
                run = lambda: fms.cluster(X, w.h, w.tol, w.max_iter, workspace=ws, precision=prec,
                                          all_seeds=True, max_modes=X.shape[0])
                r = run()
                ms, _ = _events_ms(run, 1, flush)
                st = fms.cluster(X, w.h, w.tol, w.max_iter, workspace=ws, precision=prec,
                                 all_seeds=True, max_modes=X.shape[0], profile=True).stats
                allr[prec] = {"ms": ms, "n_modes": r.stats["n_modes"],
                              "iterations": r.stats["iterations"], "evals": r.stats["evals"],
                              "fp32_step_ms": st["step_kernel_ms"],
                              "coarse_step_ms": st["coarse_kernel_ms"],
                              "coarse_evals": st["coarse_evals"], "fp32_evals": st["step_evals"],
                              "_r": r}
            rt, rf = allr["tensor"].pop("_r"), allr["fp32"].pop("_r")
            mt, mf = rt.modes.double(), rf.modes.double()
            dmat = torch.cdist(mt, mf)
            near = dmat.min(dim=1)
            matched = int((near.values <= 1e-3 * w.h).sum().item())
            # labels: a point whose tensor-path mode is matched must carry the
            # fp32-path label of that mode
            lt, lf = rt.labels.long(), rf.labels.long()
            ok_mode = near.values <= 1e-3 * w.h
            have = ok_mode[lt]
            same = int((near.indices[lt][have] == lf[have]).sum().item())
            allr["accuracy_tensor_vs_fp32"] = {
                "modes_tensor": int(mt.shape[0]), "modes_fp32": int(mf.shape[0]),
                "tensor_modes_matched_within_1e-3h": matched,
                "max_mode_diff_over_h": float(near.values.max().item() / w.h),
                "points_of_matched_modes": int(have.sum().item()),
                "same_label_among_them": same}
            allr["speedup_tensor_over_fp32"] = allr["fp32"]["ms"] / allr["tensor"]["ms"]
            line["all_seeds"] = allr
    elif args.workload == "pixels_rgb":
        # N1: RGB image segmentation, 512^2 and 1024^2 pixels (the paper's image workload)
        line.update({"metric": "ms per RGB image segmentation (labels for every pixel)",
                     "unit": "ms"})
        for side in (512, 1024):
            w = fi.pixels_rgb(seed=side, height=side, width=side)
            Xh = torch.from_numpy(w.X).pin_memory()
            X = Xh.cuda()
            n = X.shape[0]
            ws = fms.Workspace(fms.workspace_size(n, 3), X.device)
            lab_h = torch.empty(n, dtype=torch.int32).pin_memory()
            run = lambda: fms.cluster(X, w.h, w.tol, w.max_iter, workspace=ws)
            r = run()
            ms, _ = _events_ms(run, max(5, min(50, args.steps)), flush)

            ws_h = fms.Workspace(int(fms._lib.fms_cluster_host_workspace_size(
                n, 3, 256, ctypes.byref(fms.make_options()))), X.device)
            modes_h = torch.empty((256, 3), dtype=torch.float32).pin_memory()

            def e2e():   # host buffers through fms_cluster_host
                fms.cluster_host(Xh, w.h, w.tol, w.max_iter, workspace=ws_h,
                                 out=(modes_h, lab_h, None))
            for _ in range(3):
                e2e()
            e2e_ms, _ = _events_ms(e2e, max(5, min(50, args.steps)), flush)
            line[f"{side}x{side}"] = {
                "n": n, "ms": ms, "e2e_ms": e2e_ms, "n_modes": r.stats["n_modes"],
                "workspace_mb": r.stats["workspace_bytes"] / 2**20,
                "device_mb_total": (r.stats["workspace_bytes"] + n * 3 * 4 + n * 8) / 2**20,
                "evals": r.stats["evals"], "rounds": r.stats["rounds"]}
        line["value"] = line["1024x1024"]["ms"]
    elif args.workload == "flat_3d":
        # N2: the flat (uniform) kernel of Eq. 12-15 on the 200K-point 3-D workload
        w = fi.paper_3d()
        X = torch.from_numpy(w.X).cuda()
        n = X.shape[0]
        line.update({"metric": "ms per 200K-point clustering, flat kernel (Eq. 12-15)",
                     "unit": "ms"})
        for kern in ("flat", "gaussian"):
            ws = fms.Workspace(fms.workspace_size(n, 3, kernel=kern), X.device)
            run = lambda: fms.cluster(X, w.h, w.tol, w.max_iter, workspace=ws, kernel=kern)
            r = run()
            ms, _ = _events_ms(run, max(5, min(100, args.steps)), flush)
            st = fms.cluster(X, w.h, w.tol, w.max_iter, workspace=ws, kernel=kern,
                             profile=True).stats
            line[kern] = {"ms": ms, "n_modes": r.stats["n_modes"], "rounds": r.stats["rounds"],
                          "evals": r.stats["evals"],
                          "round_kernel_evals_per_s": st["round_evals"] / max(st["round_kernel_ms"], 1e-9) * 1e3,
                          "phase_ms": st["phase_ms"]}
        line["value"] = line["flat"]["ms"]
    elif args.workload == "frames_3d":
        # N3: a frame sequence (8 frames x 200K points, 20 drifting blobs) with the
        # paper's seed-count carry-over (H = 32) against starting every frame afresh
        frames = fi.drifting_frames(seed=0, frames=8, n=200_000, k=10, sigma=2.0, box=200.0)
        Fx = torch.from_numpy(np.stack(frames)).cuda()
        line.update({"metric": "ms per frame, 8 frames x 200K points (3-D, 10 drifting blobs), "
                               "768 initial seeds, seed-count carry-over",
                     "unit": "ms"})
        for label, kw in (("carry_H32", dict(H=32.0, n_initial=768)),
                          ("fresh_each_frame", dict(H=32.0, n_initial=768, fresh=True))):
            fresh = kw.pop("fresh", False)
            ws = fms.Workspace(fms.workspace_size(Fx.shape[1], 3), Fx.device)
            if fresh:
                run = lambda: [fms.cluster(Fx[f], 5.0, 5e-3, 300, n_initial=768, workspace=ws)
                               for f in range(Fx.shape[0])]
            else:
                run = lambda: fms.cluster_frames(Fx, 5.0, 5e-3, 300, workspace=ws, **kw)
            r = run()
            ms, _ = _events_ms(run, max(3, min(20, args.steps)), flush)
            rec = {"ms_per_frame": ms / Fx.shape[0]}
            if not fresh:
                rec["seed_counts"] = r.seed_counts
                rec["n_modes"] = [int(m.shape[0]) for m in r.modes]
            line[label] = rec
        line["value"] = line["carry_H32"]["ms_per_frame"]
    elif args.workload == "cosine_embed":
        # N4: the cosine metric on direction data (200K unit-normal-like points
        # in 3-D, 200K embedding-like points in 16-D), against the Euclidean
        # metric on the same points normalised beforehand
        line.update({"metric": "ms per 200K-point clustering, cosine metric", "unit": "ms"})
        for d, k, spread, h, ang in ((3, 20, 0.04, 0.12, 0.5), (16, 32, 0.04, 0.25, 0.9)):
            w = fi.directional_blobs(seed=100 + d, k=k, d=d, per=200_000 // k, spread=spread,
                                     h=h, min_angle=ang)
            X = torch.from_numpy(w.X).cuda()
            U = X / X.norm(dim=1, keepdim=True)
            n = X.shape[0]
            rec = {"n": n, "k": k, "h_chord": h}
            for metric, pts in (("cosine", X), ("euclidean_on_normalised", U)):
                mname = "cosine" if metric == "cosine" else "euclidean"
                ws = fms.Workspace(fms.workspace_size(n, d, metric=mname), X.device)
                outs = (torch.empty((n, d), device="cuda"),
                        torch.empty(n, dtype=torch.int32, device="cuda"),
                        torch.empty(n, device="cuda"))
                run = lambda: fms.cluster(pts, w.h, w.tol, w.max_iter, workspace=ws, metric=mname,
                                          out=outs)
                run()
                ms, _ = _events_ms(run, max(5, min(50, args.steps)), flush)
                r = run()   # stats of a timed-form call (the CUDA-graph form from the second on)
                rec[metric] = {"ms": ms, "n_modes": r.stats["n_modes"], "rounds": r.stats["rounds"],
                               "evals": r.stats["evals"],
                               "evals_per_s": r.stats["evals"] / (ms * 1e-3),
                               "graph": r.stats["graph"]}
            line[f"d{d}"] = rec
        line["value"] = line["d3"]["cosine"]["ms"]
    elif args.workload == "step_wide":
        # one update of every point as a seed: the coarse tensor-core step vs the FP32 step
        peaks = measured_peaks()
        # the tcgen05 rate measured on this device (completed MMAs, N = 128, one
        # issuing thread per SM) at the maximum SM clock, as the tensor roofline
        tcr = fms.probe_tensor_rates()
        smx = peaks.get("sm_max_mhz") or 2070.0
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        tc_peak = tcr["n128"]["one_issuer"] * sms * smx * 1e6 / 1e12
        line["tcgen05_flop_per_clk_sm"] = {k: v["one_issuer"] for k, v in tcr.items()}
        line["tcgen05_peak_tflops"] = tc_peak
        for d in (16, 32):
            w = fi.embedding_32d(d=d)
            X = torch.from_numpy(w.X).cuda()
            n = X.shape[0]
            rec = {"n": n, "m": n, "evals": n * n}
            for kind, fn, size in (("coarse", fms.mean_shift_step_coarse, fms._lib.fms_coarse_step_workspace_size),
                                   ("fp32", fms.mean_shift_step, fms._lib.fms_step_workspace_size)):
                ws = fms.Workspace(int(size(n, d, n)), X.device)
                run = lambda: fn(X, X, w.h, workspace=ws)
                run()
                ms, _ = _events_ms(run, max(3, min(10, args.steps)), flush)
                rec[kind] = {"ms": ms, "evals_per_s": n * n / (ms * 1e-3)}
            dpad = 16 if d <= 16 else 32
            # issued MMA work per seed-point pair: S = three BF16 split products
            # (K = dpad each) plus the 16-wide norm block; P [Xh | Xl | 1 ..]
            # (N = 2 dpad + 16)
            mma_flops = 2.0 * (3 * dpad + 16 + 2 * dpad + 16) * n * n
            alg_flops = (4.0 * d + 2) * n * n
            tf = peaks.get("bf16_tflops")
            rec["coarse"]["mma_tflops"] = mma_flops / (rec["coarse"]["ms"] * 1e-3) / 1e12
            rec["coarse"]["algorithmic_tflops"] = alg_flops / (rec["coarse"]["ms"] * 1e-3) / 1e12
            if tf:
                rec["coarse"]["mma_frac_of_measured_bf16"] = rec["coarse"]["mma_tflops"] / tf
            if tc_peak:
                rec["coarse"]["mma_frac_of_measured_tcgen05"] = rec["coarse"]["mma_tflops"] / tc_peak
            rec["speedup_coarse_over_fp32"] = rec["fp32"]["ms"] / rec["coarse"]["ms"]
            line[f"d{d}"] = rec
        line["metric"] = "ms per update of 65,536 seeds against 65,536 points"
        line["unit"] = "ms"
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="fms", choices=["fms", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-all-seeds", action="store_true",
                    help="skip the all-seeds (Alg. 1) record of the headline line")
    ap.add_argument("--workload", default="paper_3d",
                    choices=["paper_3d", "all_seeds_3d", "batched_16d", "unrolled_16d",
                             "embedding_32d", "step_wide", "pixels_rgb", "flat_3d", "frames_3d",
                             "cosine_embed"],
                    help="paper_3d is the headline line; the others print one line of "
                         "their own measurements")
    ap.add_argument("--kernel-probe", type=int, default=0, metavar="M",
                    help="only run fms_mean_shift_step with M seeds on the workload's points "
                         "(a small case for ncu captures of ms_step), then exit")
    ap.add_argument("--oracle-sample-only", type=float, default=0.0, metavar="SECONDS",
                    help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_sample_only > 0:
        ms, runs, _ = run_oracle_sample(make_input(0), seconds=args.oracle_sample_only)
        print(json.dumps({"ms": ms, "runs": runs}))
        return
    if args.kernel_probe:
        kernel_probe(args.kernel_probe)
        return
    if args.workload != "paper_3d":
        bench_extra(args)
        return
    if args.impl == "reference":
        bench_reference(args)
    else:
        bench_fms(args)


if __name__ == "__main__":
    main()
