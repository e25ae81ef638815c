"""Benchmark: RK4 steps x trajectories / s of TD-aGW propagation, low-rank vs full kernel.

Workload (one trajectory, the paper's MoS2 kernel size, Appendix A): four-band lattice
model on a 36 x 36 k-grid, N = Nb^2 Nk = 20736, dense complex64 kernel of 3.44 GB, its
randomised truncated SVD at rank 1024 (~5%, Sec. "SVD acceleration"), Gaussian * cos
pulse, RK4 at dt = 0.2 a.u.  One bench step = one RK4 step (four kernel contractions,
commutators, stage updates and the observables of the new state).

Our arm (default): the CUDA library through its C ABI.  `value` is the low-rank path's
steps/s with inputs resident on the device; the full-kernel path is timed on the same GPU
and reported beside it.  `--impl reference` times the FP64 CPU oracle (the only other
program here that computes this) on the host cores, on a bounded prefix of the same
trajectory.

Secondary legs, run after the headline region and reported in the same JSON line (each
also alone with `--leg NAME`): `batched_sweep` (256 uneven trajectories: FP32, split-FP16
tensor cores, dense), `precision_study` (N = 36864, rank 2048, B = 64), `adjoint`
(checkpointed forward + backward sweep), `channel_wise` (the channel-wise compressed
kernel at the mos2 size), `angle_hhg` (60 field directions, then their HHG spectra),
`channel_wise_sweep` (the field sweep with the channel-wise kernel, batched) and
`kdiag_split` (the two readings of K^diag on the direct + exchange kernel).

Accuracy (same JSON line): P(t) of the headline run against the FP64 oracle over a
200-step prefix, with the GPU's own rank-1024 factors (the same-factor error, held to 1e-5)
and against the oracle's full kernel (the truncation error of rank 1024 on this kernel,
which is above 1e-4); `accuracy_qualified` gives the speed-up over the full kernel of the
channel-wise form, which stays within 1e-4 of the full kernel.

Multi-GPU (torchrun, one rank per GPU): independent replicas, one trajectory per rank
(the single-trajectory path has no exchange step), value = sum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

METRIC = ("RK4 steps x trajectories / s (rank-1024 low-rank kernel vs full kernel, same GPU, "
          "single trajectory; P(t) within 1e-5 of the FP64 oracle with the same factors)")
UNIT = "steps*traj/s"
CLOCK_WINDOW_S = 1.5
# FP32 (non-tensor) peak of the GPU: 152 SMs x 128 FP32 lanes x 2 FLOP x 2.07 GHz
FP32_SIMT_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--full-steps", type=int, default=200)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--leg", choices=["sweep", "precision", "adjoint", "tc_mid", "channel", "channel_sweep",
                                      "channel_batched", "angle_hhg", "kblock"], default=None,
                    help="run one secondary leg alone and print its JSON (profiling runs)")
    ap.add_argument("--leg-steps", type=int, default=None, help="step count of the --leg run")
    return ap.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The largest per-rank value of a timing (one all-reduce); x itself on one rank."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(ws: int, units_per_rank: float, seconds: float) -> float:
    """Whole-job throughput of ws independent replicas timed over the slowest rank."""
    return ws * units_per_rank / seconds


# ---------------------------------------------------------------- clocks ------------

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def _profiled_traffic(stages: int):
    """DRAM bytes of one persistent launch from the committed ncu summary, scaled by the
    stages the launch runs; None if the kernel sources changed since the capture."""
    import hashlib
    import re
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2502_05635_gb300", "csrc")
    for f in ("lr_persistent.cu", "persist.cuh", "stage.cuh"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    # the device helpers of the common header (everything before its host-side sections)
    common = open(os.path.join(csrc, "common.cuh"), "rb").read()
    h.update(common.split(b"// " + b"-" * 66 + b" host model")[0])
    try:
        txt = open(os.path.join(ROOT, "profiles", "lr_persistent_kernel_mos2size.md")).read()
    except OSError:
        return None
    sha = re.search(r"source_sha1:\s*([0-9a-f]+)", txt)
    per = re.search(r"dram_bytes_per_stage:\s*(\d+)", txt)
    if not sha or not per or sha.group(1) != h.hexdigest():
        return None
    return int(per.group(1)) * stages


def workload_config(n_gpus: int) -> dict:
    """The headline workload's `config`, the same on both arms."""
    w = wl.mos2size_nb4_l36()
    return {"workload": w.name, "N": w.model.N, "Nk": w.model.Nk, "Nb": w.model.Nb, "rank": w.rank,
            "B": 1, "dt": w.dt, "parallelism": f"replicas x{n_gpus}",
            "l2": "inputs larger than L2 (low-rank factors 340 MB, dense kernel 3.44 GB)"}


# ---------------------------------------------------------------- oracle leg --------

def oracle_lowrank_rate(max_seconds: float, max_steps: int, warmup: int = 1):
    """The FP64 oracle's low-rank RK4 on the same workload (seeded rank-1024 factors), on
    the host cores: steps/s over a bounded prefix, after `warmup` untimed steps."""
    from oracle import lowrank as olr
    from oracle import model as om
    from oracle import propagate as op
    w = wl.mos2size_nb4_l36()
    mdl = om.Model(w.model)
    U, S, V, d = wl.random_factors(mdl.N, w.rank, seed=17)
    apply = lambda v: olr.apply_lowrank(d, U, S, V, v)  # noqa: E731
    s = op.half_step_samples(w.pulses[0], w.dt, max_steps)
    for _ in range(max(1, warmup)):                     # warm caches
        op.rk4(mdl, apply, s, w.dt, 1)
    n, t0 = 0, time.perf_counter()
    x = None
    while n < max_steps and time.perf_counter() - t0 < max_seconds:
        _, x = op.rk4(mdl, apply, s[2 * n:], w.dt, 1, x0=x)
        n += 1
    dt = time.perf_counter() - t0
    return n / dt, n, dt


def oracle_prefix(mdl, apply, samples, dt, max_steps: int, max_seconds: float):
    """The oracle's RK4 (Eq. tdagw) step by step from rho0 until max_steps or max_seconds:
    (observables rows 0..n, n, seconds)."""
    from oracle import propagate as op
    rows, x, n = [], None, 0
    t0 = time.perf_counter()
    while n < max_steps and (n == 0 or time.perf_counter() - t0 < max_seconds):
        o, x = op.rk4(mdl, apply, samples[2 * n:], dt, 1, x0=x)
        if n == 0:
            rows.append(o[0])
        rows.append(o[1])
        n += 1
    return np.array(rows), n, time.perf_counter() - t0


def accuracy_vs_oracle(tg, ctx, w, field, max_steps=200, max_seconds=45.0):
    """P(t) of the headline run checked against the FP64 oracle over a prefix: the oracle's
    low-rank RK4 with the GPU's own rank-1024 factors (tdagw_get_factors) and its full-kernel
    RK4 (FFT form of the dense K).  Also returns the oracle's low-rank rate as the CPU
    baseline (the same run)."""
    from oracle import kernel as ok
    from oracle import lowrank as olr
    from oracle import model as om
    from oracle import propagate as op
    mdl = om.Model(w.model)
    U, S, V, d = tg.tdagw_get_factors(ctx.h)
    s = op.half_step_samples(w.pulses[0], w.dt, max_steps)
    ref_lr, n, secs = oracle_prefix(mdl, lambda v: olr.apply_lowrank(d, U, S, V, v), s, w.dt,
                                    max_steps, max_seconds)
    del U, V
    kfft = ok.fft_applier(mdl)
    ref_full, _, _ = oracle_prefix(mdl, kfft, s, w.dt, n, 1e9)
    tg.tdagw_propagate(ctx.h, field, [n], w.dt, tg.LOWRANK, tg.FLAG_RESET)
    gpu_lr = tg.tdagw_observables(ctx.h)
    tg.tdagw_propagate(ctx.h, field, [n], w.dt, tg.FULL, tg.FLAG_RESET)
    gpu_full = tg.tdagw_observables(ctx.h)
    e = lambda a, b: op.rel_l2(a[:, 0], b[:, 0])  # noqa: E731
    trunc = e(ref_lr, ref_full)
    out = {"steps_compared": n, "observable": "P_x(t), relative L2 over the prefix",
           "gpu_lowrank_vs_oracle_same_factors": e(gpu_lr, ref_lr),
           "truncation_oracle_lowrank_vs_oracle_full": trunc,
           "gpu_lowrank_vs_oracle_full": e(gpu_lr, ref_full),
           "gpu_full_vs_oracle_full": e(gpu_full, ref_full),
           "gpu_lowrank_vs_gpu_full": e(gpu_lr, gpu_full),
           "tolerance_same_factors": 1e-5}
    out["within_tolerance_same_factors"] = out["gpu_lowrank_vs_oracle_same_factors"] <= 1e-5
    out["within_1e-4_of_full_kernel"] = out["gpu_lowrank_vs_oracle_full"] <= 1e-4
    cpu = {"value": n / secs, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
           "sample": f"first {n} RK4 steps of the same trajectory on the FP64 oracle, low-rank apply "
                     f"with the GPU's rank-{w.rank} factors ({secs:.1f} s; the accuracy reference)"}
    return out, cpu


def run_reference(a):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    budget = 150.0
    per_step = budget / max(1, a.steps + a.warmup)
    warm = max(1, min(a.warmup, 3))
    rate, n, secs = oracle_lowrank_rate(min(120.0, per_step * a.steps), a.steps, warm)
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": a.gpus,
            "steps": n, "warmup": warm, "ms_per_step": 1e3 / rate, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128 (fp64)", "data": "synthetic",
            "config": workload_config(a.gpus),
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"first {n} RK4 steps of the mos2size_nb4_l36 trajectory, "
                                       f"low-rank apply with seeded rank-1024 factors ({secs:.1f} s)"},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _time_propagate(tg, torch, stream, ctx, fields, steps, dt, mode, flags):
    """Device time (ms) of one batched propagate after a short warm-up run."""
    tg.tdagw_propagate(ctx.h, fields, [min(8, s) for s in steps], dt, mode, flags)
    tg.tdagw_sync(ctx.h)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    tg.tdagw_propagate(ctx.h, fields, list(steps), dt, mode, flags)
    e1.record(stream)
    torch.cuda.synchronize()
    tg.tdagw_sync(ctx.h)
    return e0.elapsed_time(e1)


def _rel_errs(a, b, steps):
    errs = []
    for j, T in enumerate(steps):
        x, y = a[:T + 1, j, 0], b[:T + 1, j, 0]
        errs.append(float(np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-300)))
    return {"max": max(errs), "median": float(np.median(errs))}


def bench_batched(tg, torch, stream, sh, tflops_peak):
    """Field sweep: 256 trajectories of uneven length (500-4000 steps) in one launch,
    two-band 24 x 24 model (N = 2304), rank 256: low-rank FP32 (SIMT), low-rank split-FP16
    on the tensor cores, and the dense kernel."""
    w = wl.sweep_nb2_l24()
    ctx = tg.Context(w.model, tg.C64, stream=sh)
    tg.tdagw_compress_svd(ctx.h, w.rank, w.oversample, w.power_iters, wl.SKETCH_SEED, precision=1)
    fields = [tg.make_field(p) for p in w.pulses]
    total = int(sum(w.steps))
    out = {"workload": "sweep_nb2_l24", "N": w.model.N, "B": w.B, "rank": w.rank,
           "traj_steps": total, "max_steps": int(max(w.steps))}
    obs = {}
    legs = (("lowrank", tg.LOWRANK, tg.FLAG_RESET),
            ("lowrank_split_f16", tg.LOWRANK, tg.FLAG_RESET | tg.FLAG_SPLIT_F16),
            ("full", tg.FULL, tg.FLAG_RESET))
    for name, mode, flags in legs:
        ms = _time_propagate(tg, torch, stream, ctx, fields, w.steps, w.dt, mode, flags)
        obs[name] = tg.tdagw_observables(ctx.h, B=w.B)
        flops = total * 4 * (2 * 8 * w.model.N * w.rank if mode == tg.LOWRANK else 8 * w.model.N ** 2)
        out[name] = {"value": total / (ms * 1e-3), "unit": "traj*steps/s", "ms": ms,
                     "algorithmic_tflops": flops / (ms * 1e-3) / 1e12}
    sp = out["lowrank_split_f16"]
    # tensor-pipe fractions of the split-FP16 leg: algorithmic complex FLOPs, and the
    # executed FP16 MMA FLOPs (three split products per term)
    sp["tensor_frac_algorithmic"] = sp["algorithmic_tflops"] / tflops_peak
    sp["tensor_frac_executed"] = 3 * sp["algorithmic_tflops"] / tflops_peak
    out["speedup_lowrank_vs_full"] = out["lowrank"]["value"] / out["full"]["value"]
    out["speedup_split_f16_vs_full"] = sp["value"] / out["full"]["value"]
    out["p_rel_err_split_f16_vs_fp32_lowrank"] = _rel_errs(obs["lowrank_split_f16"], obs["lowrank"], w.steps)
    # the accuracy the speed-ups are quoted at: each low-rank run against the dense kernel
    out["p_rel_err_lowrank_vs_full"] = _rel_errs(obs["lowrank"], obs["full"], w.steps)
    out["p_rel_err_split_f16_vs_full"] = _rel_errs(obs["lowrank_split_f16"], obs["full"], w.steps)
    ctx.close()
    return out


def precision_oracle_job(path: str, steps: int):
    """FP64 oracle run of one precision-study trajectory with the factors saved at `path`
    (the GPU's own; run in a spawned process beside the GPU legs): observables rows."""
    from oracle import lowrank as olr
    from oracle import model as om
    from oracle import propagate as op
    z = np.load(path)
    w = wl.prec_nb4_l48()
    mdl = om.Model(w.model)
    U, V = z["U"].astype(np.complex128), z["V"].astype(np.complex128)
    S, d, b = z["S"].astype(np.float64), z["d"].astype(np.complex128), int(z["b"])
    pulse = w.pulses[b]
    t0 = time.perf_counter()
    ref, _ = op.rk4(mdl, lambda v: olr.apply_lowrank(d, U, S, V, v), op.half_step_samples(pulse, w.dt, steps),
                    w.dt, steps, direction=(pulse.dir_x, pulse.dir_y))
    return ref, time.perf_counter() - t0


def bench_precision(tg, torch, stream, sh, hbm, split_steps=300, fp32_steps=30, full_steps=6, oracle_steps=100):
    """The precision study: four-band 48 x 48 model (N = 36864), rank 2048 from the GPU's
    randomised SVD (oversampling 64, two power iterations, FP64 orthogonalisation; setup
    outside the timed regions), B = 64 trajectories of the sweep distributions.  Timed:
    split-FP16 (tensor cores, Kahan-compensated RK4), plain FP32 and the dense kernel.
    Accuracy: split-FP16 and FP32 (with and without compensation) against each other over
    the FP32 run, and against the FP64 oracle with the same factors over an `oracle_steps`
    prefix of the widest pulse, computed in a spawned process while later legs run; returns
    (result, finish) where finish() joins the oracle and fills in its errors."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import tempfile
    w = wl.prec_nb4_l48()
    ctx = tg.Context(w.model, tg.C64, stream=sh)
    t0 = time.perf_counter()
    tg.tdagw_compress_svd(ctx.h, w.rank, w.oversample, w.power_iters, wl.SKETCH_SEED, precision=1)
    tg.tdagw_sync(ctx.h)
    setup = time.perf_counter() - t0
    fields = [tg.make_field(p) for p in w.pulses]
    N, r, B = w.model.N, w.rank, w.B
    out = {"workload": "prec_nb4_l48", "N": N, "B": B, "rank": r,
           "factors": f"GPU randomised SVD (p = {w.oversample}, q = {w.power_iters}), split-FP16 tiles",
           "setup_s": setup}
    obs = {}
    legs = (("lowrank_split_f16", tg.LOWRANK, tg.FLAG_RESET | tg.FLAG_SPLIT_F16, split_steps),
            ("lowrank", tg.LOWRANK, tg.FLAG_RESET, fp32_steps),
            ("full", tg.FULL, tg.FLAG_RESET, full_steps))
    for name, mode, flags, T in legs:
        ms = _time_propagate(tg, torch, stream, ctx, fields, [T] * B, w.dt, mode, flags)
        obs[name] = tg.tdagw_observables(ctx.h, B=B)
        per_stage = 2 * N * r * 8 if mode == tg.LOWRANK else N * N * 8
        gbs = 4 * T * per_stage / (ms * 1e-3) / 1e9
        out[name] = {"value": T * B / (ms * 1e-3), "unit": "traj*steps/s", "steps": T, "ms": ms,
                     "factor_gbs": gbs, "hbm_frac": gbs / hbm}
    out["speedup_split_f16_vs_full"] = out["lowrank_split_f16"]["value"] / out["full"]["value"]
    out["speedup_split_f16_vs_fp32_lowrank"] = out["lowrank_split_f16"]["value"] / out["lowrank"]["value"]
    # accuracy runs over the oracle prefix (untimed)
    T = max(fp32_steps, oracle_steps)
    runs = {}
    for name, flags in (("split_f16_kahan", tg.FLAG_RESET | tg.FLAG_SPLIT_F16),
                        ("split_f16_plain", tg.FLAG_RESET | tg.FLAG_SPLIT_F16 | tg.FLAG_NO_KAHAN),
                        ("fp32_kahan", tg.FLAG_RESET), ("fp32_plain", tg.FLAG_RESET | tg.FLAG_NO_KAHAN)):
        tg.tdagw_propagate(ctx.h, fields, [T] * B, w.dt, tg.LOWRANK, flags)
        runs[name] = tg.tdagw_observables(ctx.h, B=B)
    out["p_rel_err_split_f16_vs_fp32"] = _rel_errs(runs["split_f16_kahan"], runs["fp32_kahan"], [T] * B)
    b = int(np.argmax([p.sigma for p in w.pulses]))
    U, S, V, d = tg.tdagw_get_factors(ctx.h)
    ctx.close()
    tmp = tempfile.NamedTemporaryFile(suffix=".npz", delete=False)
    tmp.close()
    np.savez(tmp.name, U=U.astype(np.complex64), V=V.astype(np.complex64), S=S, d=d, b=b)
    del U, V
    pool = cf.ProcessPoolExecutor(max_workers=1, mp_context=mp.get_context("spawn"))
    fut = pool.submit(precision_oracle_job, tmp.name, oracle_steps)

    def finish():
        try:
            ref, secs = fut.result()
        finally:
            pool.shutdown()
            os.unlink(tmp.name)
        n = oracle_steps
        acc = {"trajectory": b, "steps": n, "oracle_s": secs}
        for name, o in runs.items():
            acc[name] = float(np.linalg.norm(o[:n + 1, b, 0] - ref[:, 0]) / np.linalg.norm(ref[:, 0]))
        acc["within_1e-4"] = acc["split_f16_kahan"] <= 1e-4
        acc["fp32_within_1e-5"] = acc["fp32_kahan"] <= 1e-5
        out["p_rel_err_vs_fp64_oracle"] = acc
        return out
    return out, finish


def bench_adjoint(tg, torch, stream, sh, T=1000):
    """Differentiation size: two-band 36 x 36 model (N = 5184), rank 512, B = 32 equal
    lengths: the checkpointed forward and the discrete adjoint (objective 1/2 sum P_x^2),
    with the forward and the segment recomputes in FP32 and on the tensor cores (split-FP16
    factors; the reverse stages use the FP32 factors in both)."""
    w = wl.adj_nb2_l36()
    ctx = tg.Context(w.model, tg.C64, stream=sh)
    tg.tdagw_compress_svd(ctx.h, w.rank, w.oversample, w.power_iters, wl.SKETCH_SEED, precision=1)
    fields = [tg.make_field(p) for p in w.pulses]
    B = w.B
    out = {"workload": "adj_nb2_l36", "N": w.model.N, "B": B, "rank": w.rank, "steps": T}
    grads = {}
    for name, extra in (("fp32", 0), ("split_f16", tg.FLAG_SPLIT_F16)):
        ms_fwd = _time_propagate(tg, torch, stream, ctx, fields, [T] * B, w.dt, tg.LOWRANK,
                                 tg.FLAG_RESET | tg.FLAG_CHECKPOINT | extra)
        P = tg.tdagw_observables(ctx.h, B=B)
        d = np.zeros((T + 1, B, 3))
        d[:, :, 0] = P[:, :, 0]
        t0 = time.perf_counter()
        gE, gp = tg.tdagw_adjoint(ctx.h, d, T, B)
        s_adj = time.perf_counter() - t0
        grads[name] = gE
        out[name] = {"forward_checkpointed": {"value": T * B / (ms_fwd * 1e-3), "unit": "traj*steps/s", "ms": ms_fwd},
                     "adjoint": {"value": T * B / s_adj, "unit": "traj*steps/s", "ms": s_adj * 1e3},
                     "forward_plus_adjoint": {"value": T * B / (ms_fwd * 1e-3 + s_adj), "unit": "traj*steps/s"},
                     "gradients_finite": bool(np.all(np.isfinite(gE)) and np.all(np.isfinite(gp)))}
    out["grad_rel_err_split_f16_vs_fp32"] = float(np.linalg.norm(grads["split_f16"] - grads["fp32"]) /
                                                  np.linalg.norm(grads["fp32"]))
    ctx.close()
    return out


def bench_tc_mid(tg, torch, stream, sh, hbm, steps=20):
    """Split-FP16 batched propagation at the four-band 36 x 36 size (N = 20736), rank 1024,
    B = 64 (seeded synthetic factors, 340 MB, larger than L2): the profiling case of the
    tensor-core kernel (a few GB on the device)."""
    w = wl.mos2size_nb4_l36()
    pulses, _ = wl.draw_pulses(64)
    ctx = tg.Context(w.model, tg.C64, stream=sh)
    U, S, V, d = wl.random_factors(w.model.N, w.rank, seed=3)
    tg.tdagw_set_factors(ctx.h, U, S, V, d)
    fields = [tg.make_field(p) for p in pulses]
    ms = _time_propagate(tg, torch, stream, ctx, fields, [steps] * 64, w.dt, tg.LOWRANK,
                         tg.FLAG_RESET | tg.FLAG_SPLIT_F16)
    gbs = 4 * steps * 2 * w.model.N * w.rank * 8 / (ms * 1e-3) / 1e9
    ctx.close()
    return {"workload": "mos2size_nb4_l36 x 64", "N": w.model.N, "B": 64, "rank": w.rank, "steps": steps,
            "value": steps * 64 / (ms * 1e-3), "unit": "traj*steps/s", "ms": ms, "factor_gbs": gbs,
            "hbm_frac": gbs / hbm}


def bench_channel_sweep(tg, torch, stream, sh):
    """The field sweep (two-band 24 x 24, N = 2304, 256 uneven trajectories) with the
    channel-wise kernel: dense diagonal channels, off-diagonal channels at rank 29 (5 % of
    Nk), in one batched launch; P(t) against the batched dense kernel."""
    w = wl.sweep_nb2_l24()
    ctx = tg.Context(w.model, tg.C64, stream=sh)
    tg.tdagw_compress_channels(ctx.h, 29, w.oversample, w.power_iters, wl.SKETCH_SEED)
    fields = [tg.make_field(p) for p in w.pulses]
    total = int(sum(w.steps))
    ms = _time_propagate(tg, torch, stream, ctx, fields, w.steps, w.dt, tg.CHANNEL, tg.FLAG_RESET)
    ch = tg.tdagw_observables(ctx.h, B=w.B)
    ms_sp = _time_propagate(tg, torch, stream, ctx, fields, w.steps, w.dt, tg.CHANNEL,
                            tg.FLAG_RESET | tg.FLAG_SPLIT_F16)
    sp = tg.tdagw_observables(ctx.h, B=w.B)
    tg.tdagw_propagate(ctx.h, fields, list(w.steps), w.dt, tg.FULL, tg.FLAG_RESET)
    full = tg.tdagw_observables(ctx.h, B=w.B)
    ctx.close()
    return {"workload": "sweep_nb2_l24, channel-wise rank 29", "N": w.model.N, "B": w.B, "traj_steps": total,
            "value": total / (ms * 1e-3), "unit": "traj*steps/s", "ms": ms,
            "p_rel_err_vs_full_gpu": _rel_errs(ch, full, w.steps),
            "split_f16": {"value": total / (ms_sp * 1e-3), "unit": "traj*steps/s", "ms": ms_sp,
                          "p_rel_err_vs_full_gpu": _rel_errs(sp, full, w.steps),
                          "p_rel_err_vs_fp32_channel": _rel_errs(sp, ch, w.steps)}}


def bench_channel(tg, torch, stream, sh, hbm, steps=1000, cmp_steps=200):
    """Channel-wise kernel at the mos2 size (four-band 36 x 36, N = 20736): dense diagonal
    channels and off-diagonal channels truncated to rank 65 by the GPU's randomised channel
    SVDs, single trajectory, one persistent launch; P(t) against the dense kernel on the
    same GPU over a prefix."""
    w = wl.mos2size_channel()
    ctx = tg.Context(w.model, tg.C64, stream=sh)
    t0 = time.perf_counter()
    tg.tdagw_compress_channels(ctx.h, w.rank, w.oversample, w.power_iters, wl.SKETCH_SEED)
    tg.tdagw_sync(ctx.h)
    setup = time.perf_counter() - t0
    ranks = tg.tdagw_get_channel_factors(ctx.h, arrays=False)
    N, Nb, Nk = ctx.N, ctx.Nb, ctx.Nk
    P = Nb * Nb
    # bytes streamed per stage: U and V of every channel, the dense diagonal channels
    per_stage = 8 * (2 * Nk * int(ranks.sum()) + P * Nk * Nk)
    field = [tg.make_field(w.pulses[0])]
    ms = _time_propagate(tg, torch, stream, ctx, field, [steps], w.dt, tg.CHANNEL, tg.FLAG_RESET)
    gbs = 4 * steps * per_stage / (ms * 1e-3) / 1e9
    tg.tdagw_propagate(ctx.h, field, [cmp_steps], w.dt, tg.CHANNEL, tg.FLAG_RESET)
    ch = tg.tdagw_observables(ctx.h)
    tg.tdagw_propagate(ctx.h, field, [cmp_steps], w.dt, tg.FULL, tg.FLAG_RESET)
    full = tg.tdagw_observables(ctx.h)
    ctx.close()
    return {"workload": "mos2size_nb4_l36_channel", "N": N, "rank_off_channels": w.rank,
            "nonzero_off_channels": int((ranks > 0).sum()), "steps": steps,
            "value": steps / (ms * 1e-3), "unit": "steps*traj/s", "ms": ms,
            "bytes_per_stage": per_stage,
            "roofline": {"bound": "hbm", "kernel": "ch_persistent_kernel", "achieved": gbs, "peak": hbm,
                         "unit": "GB/s", "frac": gbs / hbm},
            "p_rel_err_vs_full_gpu": float(np.linalg.norm(ch[:, 0] - full[:, 0]) / np.linalg.norm(full[:, 0])),
            "steps_compared": cmp_steps, "setup_s": setup}


def bench_channel_batched(tg, torch, stream, sh, hbm=6780.0, B=64, steps=60):
    """Batched propagation at the mos2 size (N = 20736) in the channel-wise form (dense
    diagonal channels, off-diagonal channels at rank 65 from the GPU's randomised channel
    SVDs) against the batched dense kernel on the same GPU: B trajectories of pulses that
    peak within the run, P(t) of every trajectory compared over the whole run.  The
    speed-up at P(t) within 1e-4 of the full kernel for the batched path."""
    w = wl.mos2size_channel()
    ctx = tg.Context(w.model, tg.C64, stream=sh)
    tg.tdagw_compress_channels(ctx.h, w.rank, w.oversample, w.power_iters, wl.SKETCH_SEED)
    fields = [tg.make_field(p) for p in wl.early_pulses(B)]
    T = [steps] * B
    ms_ch = _time_propagate(tg, torch, stream, ctx, fields, T, w.dt, tg.CHANNEL, tg.FLAG_RESET)
    ch = tg.tdagw_observables(ctx.h, B=B)
    ms_sp = _time_propagate(tg, torch, stream, ctx, fields, T, w.dt, tg.CHANNEL,
                            tg.FLAG_RESET | tg.FLAG_SPLIT_F16)
    sp = tg.tdagw_observables(ctx.h, B=B)
    ms_full = _time_propagate(tg, torch, stream, ctx, fields, T, w.dt, tg.FULL, tg.FLAG_RESET)
    full = tg.tdagw_observables(ctx.h, B=B)
    ctx.close()
    err, err_sp = _rel_errs(ch, full, T), _rel_errs(sp, full, T)
    # factor bytes streamed per stage by the tensor-core path: split tiles of the V and U
    # segments (8 bytes per complex entry, as complex64)
    ranks = 2 * 65 * 48
    per_stage = 8 * (w.model.Nk * ranks + w.model.N * w.model.Nk)
    full_bound_s = max(8.0 * w.model.N ** 2 / (hbm * 1e9), 8.0 * w.model.N ** 2 * B / (FP32_SIMT_TFLOPS * 1e12))
    return {"workload": "mos2size_nb4_l36, channel-wise rank 65, early pulses", "N": w.model.N, "B": B,
            "steps": steps,
            "channel_wise": {"value": B * steps / (ms_ch * 1e-3), "unit": "traj*steps/s", "ms": ms_ch,
                             "speedup_vs_full": ms_full / ms_ch, "p_rel_err_vs_full_gpu": err},
            "channel_wise_split_f16": {"value": B * steps / (ms_sp * 1e-3), "unit": "traj*steps/s", "ms": ms_sp,
                                       "speedup_vs_full": ms_full / ms_sp, "p_rel_err_vs_full_gpu": err_sp,
                                       "factor_gbs": 4 * steps * per_stage / (ms_sp * 1e-3) / 1e9,
                                       "p_rel_err_vs_fp32_channel": _rel_errs(sp, ch, T)},
            "full": {"value": B * steps / (ms_full * 1e-3), "unit": "traj*steps/s", "ms": ms_full},
            # the fastest any FP32 (non-tensor) dense step could be on this GPU: K streamed at
            # the measured copy peak, or 8 N^2 B FLOPs at the FP32 SIMT peak, whichever is
            # slower; the split-FP16 channel-wise speed-up against that bound
            "full_fp32_bound_ms": 4 * steps * full_bound_s * 1e3,
            "speedup_split_f16_vs_full_fp32_bound": 4 * steps * full_bound_s * 1e3 / ms_sp,
            "speedup_vs_full": ms_full / min(ms_ch, ms_sp),
            "p_rel_err_vs_full_gpu": err_sp if ms_sp < ms_ch else err,
            "within_1e-4": max(err["max"], err_sp["max"]) <= 1e-4}


def bench_angle_hhg(tg, torch, stream, sh, steps=2000, nfreq=512):
    """Angle-resolved HHG (Appendix C) at the mos2 size: 60 field directions over 1 .. 60
    degrees in one batched split-FP16 launch (rank 1024 from the GPU's randomised SVD), then
    the spectra of J_x up to the 9th harmonic on the GPU."""
    w = wl.angle_nb4_l36(steps=steps)
    ctx = tg.Context(w.model, tg.C64, stream=sh)
    tg.tdagw_compress_svd(ctx.h, w.rank, w.oversample, w.power_iters, wl.SKETCH_SEED, precision=1)
    fields = [tg.make_field(p) for p in w.pulses]
    ms = _time_propagate(tg, torch, stream, ctx, fields, w.steps, w.dt, tg.LOWRANK,
                         tg.FLAG_RESET | tg.FLAG_SPLIT_F16)
    obs = tg.tdagw_observables(ctx.h, B=w.B)
    omega = w.pulses[0].omega * 9.0 * np.arange(1, nfreq + 1) / nfreq
    t0 = time.perf_counter()
    spec = tg.tdagw_hhg_spectrum(obs, w.steps, w.dt, omega, component=1, stream=sh)
    hhg_s = time.perf_counter() - t0
    ctx.close()
    h3 = int(round(3 * nfreq / 9)) - 1
    return {"workload": "angle_nb4_l36", "N": w.model.N, "B": w.B, "rank": w.rank, "steps": steps,
            "value": w.B * steps / (ms * 1e-3), "unit": "traj*steps/s", "ms": ms,
            "hhg": {"nfreq": nfreq, "ms": hhg_s * 1e3, "max_order": 9},
            "third_harmonic_vs_angle_min_max": [float(spec[h3].min()), float(spec[h3].max())]}


def bench_kblock_split(tg, torch, stream, sh, hbm, steps=1000, cmp_steps=200):
    """The two readings of K^diag on the direct + exchange kernel at the mos2 size (rank
    1024 from the GPU's randomised SVD for each split): P(t) of each low-rank run against
    the dense kernel over a prefix, and the persistent launch with the k = k' blocks."""
    import dataclasses
    w = wl.mos2size_nb4_l36()
    model = dataclasses.replace(w.model, exchange=1.0)
    ctx = tg.Context(model, tg.C64, stream=sh)
    field = [tg.make_field(w.pulses[0])]
    out = {"workload": "mos2size_nb4_l36 + exchange (lambda_x = 1)", "N": ctx.N, "rank": w.rank}
    tg.tdagw_propagate(ctx.h, field, [cmp_steps], w.dt, tg.FULL, tg.FLAG_RESET)
    full = tg.tdagw_observables(ctx.h)
    for name, on in (("strict_diagonal", False), ("k_blocks", True)):
        tg.tdagw_set_kdiag_blocks(ctx.h, on)
        tg.tdagw_compress_svd(ctx.h, w.rank, w.oversample, w.power_iters, wl.SKETCH_SEED)
        tg.tdagw_propagate(ctx.h, field, [cmp_steps], w.dt, tg.LOWRANK, tg.FLAG_RESET)
        lr = tg.tdagw_observables(ctx.h)
        out[name] = {"p_rel_err_vs_full_gpu": float(np.linalg.norm(lr[:, 0] - full[:, 0]) /
                                                    np.linalg.norm(full[:, 0]))}
    # k-block persistent launch (the last split installed)
    ms = _time_propagate(tg, torch, stream, ctx, field, [steps], w.dt, tg.LOWRANK, tg.FLAG_RESET)
    P = ctx.Nb * ctx.Nb
    per_stage = 8 * (2 * ctx.N * (w.rank + (w.rank & 1)) + ctx.Nk * P * P + 2 * ctx.N)
    gbs = 4 * steps * per_stage / (ms * 1e-3) / 1e9
    out["k_blocks"].update({"value": steps / (ms * 1e-3), "unit": "steps*traj/s", "steps": steps,
                            "bytes_per_stage": per_stage,
                            "roofline": {"bound": "hbm", "kernel": "lr_persistent_kernel (k-block term)",
                                         "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm}})
    out["steps_compared"] = cmp_steps
    ctx.close()
    return out


# ---------------------------------------------------------------- our arm -----------

def run_leg(a):
    import torch

    import paper_2502_05635_gb300 as tg

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    sh = stream.cuda_stream
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs") or 6800.0
    tflops = peaks.get("bf16_tflops_sustained") or 1700.0
    n = a.leg_steps
    if a.leg == "sweep":
        out = bench_batched(tg, torch, stream, sh, tflops)
    elif a.leg == "precision":
        _, finish = bench_precision(tg, torch, stream, sh, hbm, *((n, n, n) if n else ()))
        out = finish()
    elif a.leg == "adjoint":
        out = bench_adjoint(tg, torch, stream, sh, n or 1000)
    elif a.leg == "channel":
        out = bench_channel(tg, torch, stream, sh, hbm, n or 1000)
    elif a.leg == "channel_sweep":
        out = bench_channel_sweep(tg, torch, stream, sh)
    elif a.leg == "channel_batched":
        out = bench_channel_batched(tg, torch, stream, sh, hbm, steps=n or 60)
    elif a.leg == "angle_hhg":
        out = bench_angle_hhg(tg, torch, stream, sh, n or 2000)
    elif a.leg == "kblock":
        out = bench_kblock_split(tg, torch, stream, sh, hbm, n or 1000)
    else:
        out = bench_tc_mid(tg, torch, stream, sh, hbm, n or 20)
    print(json.dumps({"leg": a.leg, **out}), flush=True)


def run_ours(a):
    import torch
    import torch.distributed as dist

    import paper_2502_05635_gb300 as tg

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    sh = stream.cuda_stream

    w = wl.mos2size_nb4_l36()
    pulse, dt = w.pulses[0], w.dt
    t_setup = time.perf_counter()
    ctx = tg.Context(w.model, tg.C64, stream=sh)
    tg.tdagw_compress_svd(ctx.h, w.rank, w.oversample, w.power_iters, wl.SKETCH_SEED)
    tg.tdagw_sync(ctx.h)
    t_setup = time.perf_counter() - t_setup
    N, r = ctx.N, w.rank
    field = [tg.make_field(pulse)]

    def timed(nsteps, mode, warm):
        tg.tdagw_propagate(ctx.h, field, [warm], dt, mode, tg.FLAG_RESET)
        tg.tdagw_sync(ctx.h)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        tg.tdagw_propagate(ctx.h, field, [nsteps], dt, mode, tg.FLAG_RESET)
        e1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(e0.elapsed_time(e1), dist if ws > 1 else None, dev)

    # low-rank path: the headline.  The clocks are sampled from before the warm-up through
    # the timed region and then through repeats of the same launch until the window spans
    # at least CLOCK_WINDOW_S, so that even a short timed region has samples under load.
    with ClockSampler(local) as clk:
        ms_lr = timed(a.steps, tg.LOWRANK, a.warmup)
        t_win = time.perf_counter()
        while time.perf_counter() - t_win < CLOCK_WINDOW_S:
            tg.tdagw_propagate(ctx.h, field, [a.steps], dt, tg.LOWRANK, tg.FLAG_RESET)
            tg.tdagw_sync(ctx.h)
    # full dense kernel, same GPU
    nf = min(a.full_steps, a.steps)
    ms_full = timed(nf, tg.FULL, 3)

    # dominant kernel timing: the low-rank contraction (V^H pass, reduce, U pass) on its own
    x = torch.zeros(N, dtype=torch.complex64, device=dev)
    y = torch.empty_like(x)
    with torch.cuda.stream(stream):
        x.normal_()
    reps = 50
    for _ in range(3):
        tg.tdagw_apply(ctx.h, tg.LOWRANK, x, y)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        tg.tdagw_apply(ctx.h, tg.LOWRANK, x, y)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_apply = e0.elapsed_time(e1) / reps
    ldu = r + (r & 1)
    bytes_apply = 8 * (2 * N * ldu) + 8 * 3 * N        # U, V, x twice, diag
    achieved_stagewise = bytes_apply / (ms_apply * 1e-3) / 1e9
    # dominant kernel of the timed region: the persistent low-rank kernel, one launch for
    # all steps (the field-table and first-observables kernels around it take microseconds)
    bytes_launch = 4 * a.steps * bytes_apply
    achieved = bytes_launch / (ms_lr * 1e-3) / 1e9
    fe0, fe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fe0.record(stream)
    for _ in range(5):
        tg.tdagw_apply(ctx.h, tg.FULL, x, y)
    fe1.record(stream)
    torch.cuda.synchronize()
    ms_apply_full = fe0.elapsed_time(fe1) / 5
    achieved_full = 8.0 * N * N / (ms_apply_full * 1e-3) / 1e9

    # end to end through the public API: the initial state and the pulse from host memory,
    # the observables rows back to host memory, all inside the host-timed region
    x0 = np.zeros(N, np.complex128)
    out = np.empty((a.steps + 1, 3))
    tg.tdagw_sync(ctx.h)
    if ws > 1:
        dist.barrier()
    t0 = time.perf_counter()
    tg.tdagw_set_state(ctx.h, x0, None, 0)
    tg.tdagw_propagate(ctx.h, field, [a.steps], dt, tg.LOWRANK, 0)
    tg.tdagw_observables(ctx.h, out)
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist if ws > 1 else None, dev)
    h2d = (x0.nbytes + 72) / a.steps
    d2h = out.nbytes / a.steps

    value = replica_rate(ws, a.steps, ms_lr * 1e-3)
    full_value = replica_rate(ws, nf, ms_full * 1e-3)
    launches = 3                    # field table, first observables row, persistent kernel
    cpu = None
    accuracy = None
    if rank == 0 and not a.no_cpu_baseline:
        accuracy, cpu = accuracy_vs_oracle(tg, ctx, w, field)
    traffic = _profiled_traffic(4 * a.steps)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    # FP16 and BF16 MMAs run at the same rate: the dense-bf16 figure, sustained (the
    # batched kernels run inside seconds-long launches)
    tflops = peaks.get("bf16_tflops_sustained") or 1700.0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_lr / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64 (fp32, Kahan-compensated state)",
        "data": "synthetic",
        "config": workload_config(ws),
        "full_kernel": {"value": full_value, "unit": UNIT, "steps": nf,
                        "ms_per_step": ms_full / nf,
                        "apply_gbs": achieved_full, "apply_ms": ms_apply_full},
        "speedup_lowrank_vs_full": value / full_value,
        "accuracy": accuracy,
        "roofline": {"bound": "hbm", "kernel": "lr_persistent_kernel",
                     "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "peak_source": peak_src,
                     "bytes_per_launch": bytes_launch, "ms_per_launch": ms_lr,
                     "bytes_per_stage": bytes_apply,
                     "traffic": traffic},
        "stagewise_apply": {"gbs": achieved_stagewise, "ms": ms_apply},
        "e2e": {"value": replica_rate(ws, a.steps, e2e_s), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": {**clk.summary(), "window": f"warm-up, timed region and repeats of the same "
                                             f"launch, >= {CLOCK_WINDOW_S} s"},
        "setup_s": t_setup,
    }
    if cpu:
        line["cpu_baseline"] = cpu
    if not a.no_batched:
        line["batched_sweep"] = bench_batched(tg, torch, stream, sh, tflops)
        prec, prec_finish = bench_precision(tg, torch, stream, sh, hbm)
        line["adjoint"] = bench_adjoint(tg, torch, stream, sh)
        line["channel_wise"] = bench_channel(tg, torch, stream, sh, hbm)
        ch = line["channel_wise"]
        # the speed-up at P(t) within 1e-4 of the full kernel: the channel-wise form
        # (Eq. svd-channel-wise) at the same size, against the same full-kernel run
        line["accuracy_qualified"] = {
            "form": "channel-wise (dense diagonal channels, off-diagonal channels rank 65)",
            "value": ch["value"], "unit": UNIT,
            "p_rel_err_vs_full_gpu": ch["p_rel_err_vs_full_gpu"], "steps_compared": ch["steps_compared"],
            "within_1e-4_of_full_kernel": ch["p_rel_err_vs_full_gpu"] <= 1e-4,
            "speedup_vs_full": ch["value"] / (nf / (ms_full * 1e-3))}
        line["channel_wise_batched"] = bench_channel_batched(tg, torch, stream, sh, hbm)
        cb = line["channel_wise_batched"]
        line["accuracy_qualified"]["batched"] = {
            "form": "channel-wise, split-FP16 segment tiles on the tensor cores",
            "value": cb["channel_wise_split_f16"]["value"], "unit": "traj*steps/s", "B": cb["B"],
            "p_rel_err_vs_full_gpu": cb["channel_wise_split_f16"]["p_rel_err_vs_full_gpu"],
            "within_1e-4": cb["channel_wise_split_f16"]["p_rel_err_vs_full_gpu"]["max"] <= 1e-4,
            "speedup_vs_full": cb["channel_wise_split_f16"]["speedup_vs_full"]}
        line["channel_wise_sweep"] = bench_channel_sweep(tg, torch, stream, sh)
        line["angle_hhg"] = bench_angle_hhg(tg, torch, stream, sh)
        line["kdiag_split"] = bench_kblock_split(tg, torch, stream, sh, hbm)
        line["precision_study"] = prec_finish()
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    elif a.leg:
        run_leg(a)
    else:
        run_ours(a)
