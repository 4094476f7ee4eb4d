#!/usr/bin/env python
"""Benchmark of the FFT Lindhard susceptibility (Eq. 9 of Wang et al.) on GB300.

One step = one whole forward call of the library on one instance of the
workload: tight-binding band tables, FP64 chemical-potential solve, spectral
generation fused into the energy FFT, the p_y FFT, the p_x FFT with the
conjugate product and inverse, the inverse p_y FFT and the inverse energy FFT
with crop and scale.  Metric: Im chi(q, w) outputs per second (whole job).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

Under torchrun (N > 1) every rank computes its own replica of the instance
(the instance does not shard; instances are independent), so per-GPU work is
fixed: "scaling": "weak", value = outputs of all ranks / max rank time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DEFAULT_WORKLOAD = "large_1024x1024x512"
FALLBACK_HBM_GBS = 6800.0
COMMON_FILES = ("fft_engine.cuh", "kernels.cuh", "lindhard_internal.h")
PASS_FILES = {  # kernel sources of each timed pass (for traffic-record staleness)
    "energy_fwd": ("k_forward.cu", "k_energy.cu", "et_tiles.cuh"),
    "py_fwd": ("k_forward.cu", "k_tma.cu", "tma.cuh", "async.cuh", "k_pruned.cu", "fft_pruned.cuh", "pr_tiles.cuh", "k_pruned_tma.cu"),
    "px_product": ("k_product.cu", "k_tma.cu", "tma.cuh", "async.cuh", "k_pruned.cu", "fft_pruned.cuh", "pr_tiles.cuh", "k_pruned_tma.cu", "k_product_pipe.cu"),
    "py_inv": ("k_inverse.cu", "k_tma.cu", "tma.cuh", "async.cuh", "k_pruned.cu", "fft_pruned.cuh", "pr_tiles.cuh", "k_pruned_tma.cu"),
    "energy_inv": ("k_inverse.cu", "k_tma.cu", "tma.cuh", "async.cuh", "k_energy.cu", "et_tiles.cuh"),
}
PASS_FILES = {k: v + COMMON_FILES for k, v in PASS_FILES.items()}
# kernel of each pass by engine variant (lindhard_plan_variants)
VARIANT_KERNELS = {
    "py_fwd": ["k_fwd_y", "k_fwd_y2", "k_fwd_y2 (12-value tiles)", "k_fwd_y_tma", "k_fwd_y_tma (12-value tiles)",
               "k_y_col_tma (forward)", "k_fwd_y2 (double-width tile)", "(unused)", "k_fwd_y_pr (pruned, 8 pairs)",
               "k_fwd_y_pr (pruned, 4 pairs)",
               "k_fwd_y_pr_tma (pruned, TMA-staged)", "k_fwd_y_pr_tma2 (pruned, TMA-staged, two CTAs per SM)"],
    "py_inv": ["k_inv_y", "k_inv_y2", "k_inv_y2 (12-value tiles)", "k_inv_y_tma", "k_inv_y_tma (12-value tiles)",
               "k_y_col_tma (inverse)", "k_inv_y2 (double-width tile)", "k_inv_y_tc (tensor cores)",
               "k_inv_y_pr (pruned, 8 pairs)", "k_inv_y_pr (pruned, 4 pairs)", "k_inv_y_pr_tma (pruned, TMA-staged)",
               "k_inv_y_pr_tma2 (pruned, TMA-staged, two CTAs per SM)"],
    "px_product": ["k_x_product", "k_x_product (12-value tiles)", "k_x_product_tma",
                   "k_x_product_tma (12-value tiles)", "k_x_product (one more CTA per SM)",
                   "k_x_product (double-width tile)", "k_x_product_pr (pruned, 8 columns)",
                   "k_x_product_pr (pruned, 4 columns)", "k_x_product_pr_tma (pruned, TMA-staged)",
                   "k_x_product_pr_pipe (pruned, pipelined)",
                   "k_x_product_pr_pipe (pruned, pipelined, twiddles in shared memory)"],
    "energy_inv": ["k_inv_energy", "k_inv_energy_tma", "k_inv_energy_warp"],
}
KERNEL_NAMES = {"batch": "all passes of all instances (graph)", "energy_fwd": "k_fwd_energy", "py_fwd": "k_fwd_y", "px_product": "k_x_product",
                "py_inv": "k_inv_y", "energy_inv": "k_inv_energy", "tables": "k_setup", "mu_solve": "k_mu_sect, k_mu_halley"}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the plan-creation timing of engine variants (paired-column engine)")
    ap.add_argument("--precision", choices=["fp32", "tc"], default="fp32",
                    help="tc: grids with LINDHARD_SPLITBF16_TC (the inverse p_y pass on the tensor cores)")
    ap.add_argument("--no-tc", action="store_true",
                    help="skip the comparison with the tensor-core form (LINDHARD_SPLITBF16_TC)")
    ap.add_argument("--grid", default=None,
                    help="zones,npz,n_eps,e_max: replace the workload's grid (for profiling smaller cases)")
    ap.add_argument("--variants", default=None,
                    help="F,I,X,E: pin the engine variants of the p_y forward, p_y inverse, product and "
                         "inverse energy passes (through a tune cache file) instead of timing them, e.g. "
                         "to profile a smaller grid with the variants the full-size workload takes")
    return ap.parse_args()


def pin_variants(lh, torch, grids, spec):
    """Write the pinned variants for the grid's geometry to a fresh tune cache
    file and point LINDHARD_TUNE_CACHE at it (the autotuner uses cached
    entries as they are)."""
    vf, vi, vx, ve = (int(v) for v in spec.split(","))
    probe = lh.Plan(grids)
    s = probe.sizes[0]
    probe.close()
    key = f"{torch.cuda.get_device_name(0)}|P={s.fft_p}|N={s.N}|PE={s.fft_e}|Q={s.q_extent}"
    path = os.path.join(tempfile.mkdtemp(prefix="lindhard_pins_"), "tune.json")
    with open(path, "w") as f:
        json.dump({key + "|fwd_y": vf, key + "|inv_y": vi, key + "|x_product": vx, key + "|inv_energy": ve},
                  f, indent=0)
    os.environ["LINDHARD_TUNE_CACHE"] = path


def pass_bytes(s):
    """Algorithmic HBM bytes of each pass for one instance (FP32, 8-byte
    complex): every intermediate written once and read once, counting only its
    non-redundant entries; the spectral function is generated on chip."""
    N, P, PE, Q, n_omega = s.N, s.fft_p, s.fft_e, s.q_extent, s.n_omega
    H = PE // 2 + 1
    W1, W2, W3, W4 = N * N * 2 * H, N * P * 2 * H, Q * P * H, Q * Q * H
    out = Q * Q * n_omega
    return {"energy_fwd": 8 * W1, "py_fwd": 8 * (W1 + W2), "px_product": 8 * (W2 + W3),
            "py_inv": 8 * (W3 + W4), "energy_inv": 8 * W4 + 4 * out}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def source_digest(fnames):
    """Hash of a pass's kernel sources together with the headers every kernel
    includes (FFT engine, tile configurations, shared types)."""
    h = hashlib.sha256()
    for f in tuple(fnames) + ("fft_engine.cuh", "kernels.cuh", "lindhard_internal.h"):
        with open(os.path.join(ROOT, "paper_1208_3210_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(pass_name, workload, variant):
    """DRAM bytes per launch from the committed ncu summary, or None when the
    kernel source changed since the counters were taken or the plan runs
    another engine variant of the pass than the one captured."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(p))[workload][pass_name]
    except Exception:
        return None
    if rec.get("source_sha256_16") != source_digest(PASS_FILES[pass_name]):
        return None
    if rec.get("variant", 0) != variant:
        return None
    return rec.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "", 1).isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def workload_instance(workload):
    """(band, grid, note) of the instance a CPU leg samples: the workload's own
    single instance, or the first instance of a batched workload."""
    from paper_1208_3210_gb300 import workloads as wl
    if workload.startswith("batched_"):
        inst = wl.batched_instances(int(workload.split("_")[1]))[0]
        return dict(inst["band"]), inst["grid"], f"instance 0 of {workload}"
    w = wl.WORKLOADS[workload]
    return dict(w["band"]), w["grid"], workload


def cpu_baseline(workload, seconds=15.0, seed=7):
    """The FP64 oracle (direct double sum of Eq. 9) on a bounded seeded sample
    of this workload's outputs, on all host cores."""
    import numpy as np

    import oracle
    band, grid, workload = workload_instance(workload)
    t0 = time.perf_counter()
    band["mu"] = oracle.solve_mu(band["kind"], band["t"], band["tp"], band["tpp"], band["gamma"], grid["npz"],
                                 band["filling"])
    A = oracle.spectral(band, grid)
    t_setup = time.perf_counter() - t0
    Q, n_omega = grid["q_extent"], grid["n_omega"]
    rng = np.random.default_rng(seed)

    def draw(n):
        return (rng.integers(0, Q, n).astype(np.int32), rng.integers(0, Q, n).astype(np.int32),
                rng.integers(0, n_omega, n).astype(np.int32))

    t0 = time.perf_counter()
    oracle.imchi_samples(A, grid, Q, *draw(32))
    rate = 32 / max(time.perf_counter() - t0, 1e-6)
    n = max(32, int(rate * seconds))
    lx, ly, m = draw(n)
    t0 = time.perf_counter()
    ref = oracle.imchi_samples(A, grid, Q, lx, ly, m)
    dt = time.perf_counter() - t0
    res = {"value": n / dt, "unit": "outputs/s", "cores": oracle.num_threads(), "kind": "oracle",
           "sample": f"FP64 direct double sum of Eq. 9 at {n} uniformly drawn outputs (q, w) of "
                     f"{workload} in {dt:.1f} s; A(p, e) tabulated once beforehand ({t_setup:.1f} s, untimed)"}
    res["fft_method"] = cpu_fft_method(A, grid, lx, ly, m, ref)
    res["host"] = host_cpu()
    return res


def host_cpu():
    """The host cores the CPU legs may use and the processor model."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    try:
        affinity = len(os.sched_getaffinity(0))
    except Exception:
        affinity = os.cpu_count() or 1
    return {"affinity_cores": affinity, "model": model or "unknown"}


def _host_available_bytes():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except Exception:
        pass
    return 0


def cpu_fft_method(A, grid, lx, ly, m, ref):
    """The paper's own comparison on the host (Sec. 3: the FFT method against
    the direct sum): every output by the FP64 FFT reference of oracle/
    (scipy, all host cores), timed, and checked against the direct sums at
    the sampled outputs.  Skipped when the host lacks the memory (about six
    complex128 volumes of the padded momentum grid times n_eps/2 + 1)."""
    import numpy as np

    from oracle.fft_reference import imchi_fft64
    zones, npz, n_eps, Q, n_omega = grid["zones"], grid["npz"], grid["n_eps"], grid["q_extent"], grid["n_omega"]
    N = zones * npz
    P = N if zones == 1 else N + Q // 2
    need = 6 * P * P * (n_eps // 2 + 1) * 16
    avail = _host_available_bytes()
    if avail < 1.3 * need:
        return {"unavailable": f"needs about {need / 1e9:.0f} GB of host memory, {avail / 1e9:.0f} GB available"}
    workers = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    t0 = time.perf_counter()
    out = imchi_fft64(A, grid, workers=workers)
    dt = time.perf_counter() - t0
    diff = float(np.abs(out[lx, ly, m] - ref).max() / max(np.abs(ref).max(), 1e-300))
    return {"value": Q * Q * n_omega / dt, "unit": "outputs/s", "seconds": dt, "cores": workers,
            "kind": "FP64 FFT reference of the whole output (oracle/fft_reference.py: scipy transforms, "
                    "conjugate product, inverse)",
            "max_rel_diff_vs_direct_sum": diff}


def run_reference(args):
    from paper_1208_3210_gb300.replicas import rank_info
    rank, _, world = rank_info()
    if rank != 0:
        return
    import numpy as np

    import oracle
    band, grid, _ = workload_instance(args.workload)
    band["mu"] = oracle.solve_mu(band["kind"], band["t"], band["tp"], band["tpp"], band["gamma"], grid["npz"],
                                 band["filling"])
    A = oracle.spectral(band, grid)
    Q, n_omega = grid["q_extent"], grid["n_omega"]
    rng = np.random.default_rng(11)
    t0 = time.perf_counter()
    oracle.imchi_samples(A, grid, Q, rng.integers(0, Q, 16).astype(np.int32),
                         rng.integers(0, Q, 16).astype(np.int32), rng.integers(0, n_omega, 16).astype(np.int32))
    # each step a bounded sample: about 2 s of CPU work, less when the whole
    # --steps + --warmup run would otherwise exceed about two minutes
    per_step_s = min(2.0, 120.0 / max(1, args.steps + args.warmup))
    per_step = max(1, int(16 / max(time.perf_counter() - t0, 1e-6) * per_step_s))

    def step():
        lx = rng.integers(0, Q, per_step).astype(np.int32)
        ly = rng.integers(0, Q, per_step).astype(np.int32)
        m = rng.integers(0, n_omega, per_step).astype(np.int32)
        oracle.imchi_samples(A, grid, Q, lx, ly, m)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt
    line = {"metric": "Im chi(q,w) outputs/s", "value": value, "unit": "outputs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "per_step_sample": f"{per_step} seeded outputs"},
            "cpu_baseline": {"value": value, "unit": "outputs/s", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"{per_step} uniformly drawn outputs per step, FP64 direct double sum"},
            "e2e": {"value": value, "unit": "outputs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def tensor_core_form(lh, grids, bands, out_fp32, steps, autotune, mu, stream):
    """The same call with precision LINDHARD_SPLITBF16_TC (the inverse p_y pass
    on the tensor cores): device time per call, the inverse p_y pass alone,
    and the largest difference from the FP32 SIMT result, outside the timed
    region of the FP32 form."""
    import torch
    tgrids = [dict(g, precision=lh.SPLITBF16_TC) for g in grids]
    try:
        tp = lh.Plan(tgrids, autotune=autotune)
    except Exception as exc:   # no tensor-core form for this length
        return {"unavailable": str(exc)}
    tout = torch.empty(tp.out_elems(), dtype=torch.float32, device="cuda")
    for _ in range(3):
        tp.imchi(bands, out=tout, mu_out=mu)
    tp.status()
    tp.profile(True)
    for _ in range(max(3, min(steps // 10, 50))):
        tp.imchi(bands, out=tout, mu_out=mu)
    pt = tp.pass_times()
    tp.profile(False)
    n = max(3, min(steps, 200))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(n):
        tp.imchi(bands, out=tout, mu_out=mu)
    e1.record(stream)
    torch.cuda.synchronize()
    tp.status()
    ms = e0.elapsed_time(e1) / n
    diff = float((tout - out_fp32).abs().max() / out_fp32.abs().max().clamp_min(1e-30))
    res = {"ms_per_step": ms, "value": tp.out_elems() / (ms * 1e-3), "steps": n,
           "py_inv_ms": round(pt["py_inv"][0] / max(pt["py_inv"][1], 1), 5),
           "max_rel_diff_vs_fp32": diff, "variants": tp.variants(0)}
    tp.close()
    return res


def kk_rpa_form(plan, out, steps, stream, peak, v0=0.05):
    """The Kramers-Kronig real part and chi_RPA (lindhard_kk_rpa, V_q = v0/|q|^2)
    of the instance's Im chi, both forms: device time per call, HBM bytes
    (Im chi read, Re chi and chi_RPA written) over that time, and the largest
    difference between the forms; outside the timed region of the forward call."""
    import torch
    s = plan.sizes[0]
    nbytes = 16 * s.q_extent * s.q_extent * s.n_omega
    res = {"v0_ev": v0, "bytes_per_call": nbytes}
    outs = {}
    for v, name in ((0, "tensor_core"), (1, "fp32_simt")):
        try:
            plan.kk_rpa(out, v0=v0, variant=v)
        except Exception as exc:
            res[name] = {"unavailable": str(exc)}
            continue
        n = max(3, min(steps, 200))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(n):
            r = plan.kk_rpa(out, v0=v0, variant=v)
        e1.record(stream)
        torch.cuda.synchronize()
        plan.status()
        ms = e0.elapsed_time(e1) / n
        outs[v] = r[0]
        res[name] = {"ms": ms, "gbs": nbytes / (ms * 1e-3) / 1e9, "frac_of_hbm_peak": nbytes / (ms * 1e-3) / 1e9 / peak,
                     "calls": n}
    if 0 in outs and 1 in outs:
        res["max_rel_diff_tc_vs_fp32"] = float((outs[0] - outs[1]).abs().max() / outs[1].abs().max().clamp_min(1e-30))
    return res


def thermal_form(lh, grids, bands, steps, autotune, stream, kT=0.025):
    """The finite-temperature quantities (grid quantity LINDHARD_IMCHI_T and
    LINDHARD_SQW at kT, energy FFT padded to PE >= n_eps + n_omega - 1): device
    time per call and outputs/s, outside the timed region of the T = 0 call."""
    import torch
    res = {"kT_ev": kT}
    for q, name in ((lh.IMCHI_T, "imchi_T"), (lh.SQW, "S_qw")):
        qgrids = [dict(g, quantity=q) for g in grids]
        qbands = [dict(b, kT=kT) for b in bands]
        try:
            qp = lh.Plan(qgrids, autotune=autotune)
        except Exception as exc:
            res[name] = {"unavailable": str(exc)}
            continue
        qout = torch.empty(qp.out_elems(), dtype=torch.float32, device="cuda")
        for _ in range(3):
            qp.imchi(qbands, out=qout)
        qp.status()
        n = max(3, min(steps, 200))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(n):
            qp.imchi(qbands, out=qout)
        e1.record(stream)
        torch.cuda.synchronize()
        qp.status()
        ms = e0.elapsed_time(e1) / n
        res[name] = {"ms_per_step": ms, "value": qp.out_elems() / (ms * 1e-3), "steps": n,
                     "fft_e": qp.sizes[0].fft_e, "variants": qp.variants(0)}
        qp.close()
        del qout
    return res


def backward_bytes(s):
    """Algorithmic HBM bytes of one adjoint call (lindhard_imchi_backward with
    dL/dA and dL/dtheta) on one instance, counted like pass_bytes: the
    forward energy and p_y passes again (a^, b^), w along energy and q_y, the
    two products along p_x (a^, b^ and W^ read, h^ and g^ written), the
    inverse along p_y and the inverse along energy writing dL/dA."""
    N, P, PE, Q, n_omega, n_eps = s.N, s.fft_p, s.fft_e, s.q_extent, s.n_omega, s.n_eps
    H = PE // 2 + 1
    W1, W2 = N * N * 2 * H, N * P * 2 * H
    WQ1, WQ2 = Q * Q * H, Q * P * H
    return 8 * (W1 + (W1 + W2) + WQ1 + (WQ1 + WQ2) + (W2 + WQ2 + W2) + (W2 + W1) + W1) + 4 * (Q * Q * n_omega
                                                                                          + N * N * n_eps)


def backward_form(lh, grids, bands, steps, stream, peak, autotune):
    """The adjoint (row a8): one lindhard_imchi_backward call for
    L = sum w Im chi with seeded weights, dL/dA and dL/d(t, t', t'', mu, gamma)
    both requested; device time per call, outside the timed region of the
    forward call."""
    import torch
    try:
        bp = lh.Plan(grids, backward=True, autotune=autotune)   # the forward p_y pass it repeats, tuned
    except Exception as exc:
        return {"unavailable": str(exc)}
    gen = torch.Generator(device="cuda").manual_seed(7)
    w = torch.rand(bp.out_elems(), generator=gen, device="cuda", dtype=torch.float32)
    dA = torch.empty(bp.a_elems(), dtype=torch.float32, device="cuda")
    dp = torch.zeros(5 * len(grids), dtype=torch.float64, device="cuda")
    for _ in range(3):
        bp.backward(w, bands=bands, dA=dA, dparams=dp)
    bp.status()
    n = max(3, min(steps, 20))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(n):
        bp.backward(w, bands=bands, dA=dA, dparams=dp)
    e1.record(stream)
    torch.cuda.synchronize()
    bp.status()
    ms = e0.elapsed_time(e1) / n
    byts = sum(backward_bytes(bp.sizes[i]) for i in range(len(grids)))
    res = {"ms_per_call": ms, "dA_elems_per_s": bp.a_elems() / (ms * 1e-3), "calls": n,
           "algorithmic_bytes": byts, "gbs": byts / (ms * 1e-3) / 1e9,
           "frac_of_hbm_peak": byts / (ms * 1e-3) / 1e9 / peak}
    bp.close()
    del w, dA, dp
    return res


def batched_form(lh, steps, autotune, stream, count=64):
    """The batched workload (`count` independent instances of mixed filling,
    broadening and size, one call per batch) in the plan's three batch forms:
    the persistent batch launch replayed as a graph, the same instances one
    after another on one stream, and every instance's launches on forked
    streams recorded into one graph; device time per batch, outside the timed
    region of the single-instance call."""
    import torch
    from paper_1208_3210_gb300 import workloads as wl
    grids, bands = wl.batched_workload(count)
    res = {"instances": count}
    n = max(3, min(steps, 10))
    ref = None
    for name, kw in (("plain_sequential", {}), ("persistent_graph", dict(graph=True, persistent=True)),
                     ("concurrent_graph", dict(graph=True))):
        try:
            p = lh.Plan(grids, autotune=autotune, **kw)
        except Exception as exc:
            res[name] = {"unavailable": str(exc)}
            continue
        o = torch.empty(p.out_elems(), dtype=torch.float32, device="cuda")
        for _ in range(3):
            p.imchi(bands, out=o)
        p.status()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(n):
            p.imchi(bands, out=o)
        e1.record(stream)
        torch.cuda.synchronize()
        p.status()
        ms = e0.elapsed_time(e1) / n
        res[name] = {"ms_per_batch": ms, "value": p.out_elems() / (ms * 1e-3), "steps": n}
        if ref is None:
            ref = o
        else:
            res[name]["max_rel_diff_vs_plain"] = float((o - ref).abs().max() / ref.abs().max().clamp_min(1e-30))
            del o
        p.close()
    if "ms_per_batch" in res.get("plain_sequential", {}):
        for name in ("persistent_graph", "concurrent_graph"):
            if "ms_per_batch" in res.get(name, {}):
                res[name]["speedup_vs_plain"] = res["plain_sequential"]["ms_per_batch"] / res[name]["ms_per_batch"]
    del ref
    return res


def energy_direct_form(lh, grids, bands, out_3d, steps, mu, stream):
    """The paper's own arrangement (LINDHARD_PLAN_ENERGY_DIRECT: 2D momentum
    FFTs per energy plane, the energy sum done directly per momentum
    frequency): device time per call, per-pass times, and the largest
    difference from the 3D FFT form, outside the timed region of the 3D call."""
    import torch
    try:
        dp = lh.Plan(grids, energy_direct=True)
    except Exception as exc:
        return {"unavailable": str(exc)}
    dout = torch.empty(dp.out_elems(), dtype=torch.float32, device="cuda")
    for _ in range(3):
        dp.imchi(bands, out=dout, mu_out=mu)
    dp.status()
    dp.profile(True)
    for _ in range(max(3, min(steps // 10, 50))):
        dp.imchi(bands, out=dout, mu_out=mu)
    pt = dp.pass_times()
    dp.profile(False)
    n = max(3, min(steps, 200))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(n):
        dp.imchi(bands, out=dout, mu_out=mu)
    e1.record(stream)
    torch.cuda.synchronize()
    dp.status()
    ms = e0.elapsed_time(e1) / n
    diff = float((dout - out_3d).abs().max() / out_3d.abs().max().clamp_min(1e-30))
    names = {"energy_fwd": "planes", "py_fwd": "py_fwd", "px_product": "px_fwd+energy_sum+kx_inv",
             "py_inv": "ky_inv", "energy_inv": "output"}
    res = {"ms_per_step": ms, "value": dp.out_elems() / (ms * 1e-3), "steps": n,
           "passes_ms": {names[k]: round(v[0] / max(v[1], 1), 5) for k, v in pt.items() if k in names},
           "max_rel_diff_vs_3d": diff}
    dp.close()
    return res


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    from paper_1208_3210_gb300 import replicas
    rank, local_rank, world = replicas.rank_info()
    import torch
    import torch.distributed as dist

    from paper_1208_3210_gb300 import build as lbuild
    from paper_1208_3210_gb300 import lindhard as lh
    from paper_1208_3210_gb300 import workloads as wl

    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    if rank == 0 or world == 1:
        lbuild.build()
    if world > 1:
        dist.barrier()

    batched = args.workload.startswith("batched_")
    persistent = False
    prec = lh.SPLITBF16_TC if args.precision == "tc" else lh.FP32
    if prec != lh.FP32:
        args.no_tc = True   # the timed form is the tensor-core one already
    if batched:
        # independent instances of mixed size, one graph call per step
        count = int(args.workload.split("_")[1])
        grids, bands = wl.batched_workload(count)
        grids = [dict(g, precision=prec) for g in grids]
        # FP32: the persistent batch launch (every instance's passes in one
        # launch) replayed as a graph; other precisions: graph of stream branches
        persistent = prec == lh.FP32
        plan = lh.Plan(grids, graph=True, persistent=persistent, autotune=not args.no_autotune)
        args.no_cpu_baseline = True
    else:
        w = wl.WORKLOADS[args.workload]
        band, grid = w["band"], w["grid"]
        if args.grid:
            z, npz, ne, em = args.grid.split(",")
            grid = wl.grid_params(int(z), int(npz), int(ne), float(em))
            args.workload = f"{args.workload} grid {args.grid}"
            args.no_cpu_baseline = True
        grids, bands = [dict(grid, precision=prec)], [band]
        if args.variants:
            pin_variants(lh, torch, grids, args.variants)
        plan = lh.Plan(grids, autotune=not args.no_autotune)
    s = plan.sizes[0]
    out = torch.empty(plan.out_elems(), dtype=torch.float32, device="cuda")
    mu = torch.empty(len(grids), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        plan.imchi(bands, out=out, mu_out=mu)

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x):
        return replicas.max_over_ranks(x, world, "cuda")

    for _ in range(max(3, args.warmup)):
        step()
    plan.status()

    # --- per-pass split from a short profiled run: every pass bracketed by
    # events (this perturbs the step, so it stays outside the timed region) ---
    ptimes = {}
    if not batched:
        plan.profile(True)
        for _ in range(max(3, min(args.steps // 10, 50))):
            step()
        ptimes = plan.pass_times()
        plan.profile(False)
        pb0 = pass_bytes(s)
        dom_pass = max((k for k in ptimes if k in pb0 and ptimes[k][1] > 0), key=lambda k: ptimes[k][0])

    # --- device-timed region: inputs resident; the dominant pass's events are
    # recorded live on its launch stream ---
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES")
    gpu_index = int(cvd.split(",")[local_rank]) if cvd else local_rank
    clocks = ClockSampler(gpu_index)
    time.sleep(0.3)
    if not batched:
        plan.profile(True, passes=[dom_pass])
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms_total = max_over_ranks(ev0.elapsed_time(ev1))
    dom_live = plan.pass_times() if not batched else {}
    if not batched:
        plan.profile(False)
    plan.status()

    # --- end to end through the public call: every step's result read back to
    # pinned host memory, streamed the way a caller overlaps transfers: two
    # device and host output buffers, each step's copy on a copy stream,
    # overlapped with the next step's computation ---
    host_outs = [torch.empty(plan.out_elems(), dtype=torch.float32, pin_memory=True) for _ in range(2)]
    dev_outs = [out, torch.empty_like(out)]
    # a caller repeating the call replays it as a CUDA graph (LINDHARD_PLAN_GRAPH):
    # one graph plan per output buffer, so neither records again
    e2e_plans = ([plan, lh.Plan(grids, graph=True, persistent=persistent, autotune=not args.no_autotune)] if batched else
                 [lh.Plan(grids, graph=True, autotune=not args.no_autotune) for _ in range(2)])
    for b in range(2):
        for _ in range(3):
            e2e_plans[b].imchi(bands, out=dev_outs[b], mu_out=mu)
        host_outs[b].copy_(dev_outs[b])
    torch.cuda.synchronize()
    copy_stream = torch.cuda.Stream()
    ready = [torch.cuda.Event() for _ in range(2)]
    copied = [torch.cuda.Event() for _ in range(2)]
    e2e_steps = max(3, min(args.steps, 200))
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        b = i % 2
        if i >= 2:
            stream.wait_event(copied[b])   # the copy that last read this buffer
        e2e_plans[b].imchi(bands, out=dev_outs[b], mu_out=mu)
        ready[b].record(stream)
        copy_stream.wait_event(ready[b])
        with torch.cuda.stream(copy_stream):
            host_outs[b].copy_(dev_outs[b], non_blocking=True)
        copied[b].record(copy_stream)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    barrier()
    for p_ in e2e_plans:
        p_.status()
    for p_ in e2e_plans:
        if p_ is not plan:
            p_.close()
    del dev_outs[1]

    outputs_per_step = plan.out_elems() * world
    value = replicas.whole_job_rate(plan.out_elems(), world, args.steps, ms_total * 1e-3)
    e2e_value = replicas.whole_job_rate(plan.out_elems(), world, e2e_steps, e2e_s)
    step_ms = ms_total / args.steps
    peak, peak_kind = measured_peaks()
    # kernels launched in the timed region: each step is one forward call; a
    # third multisection pass when gamma < 0.02 eV and the solve spans
    # several CTAs (more than 98 points per zone)
    launches = (sum(int(plan.sizes[i].kernels_forward)
                    + (1 if bands[i]["gamma"] < 0.02 and grids[i]["npz"] > 98 else 0)
                    for i in range(len(grids))) + (1 if batched and persistent else 0)) * args.steps
    if batched:
        # concurrent instances: no per-pass split, the batch as one unit
        pipeline_bytes = sum(sum(pass_bytes(plan.sizes[i]).values()) for i in range(len(grids)))
        dom, pb, dom_ms, traffic = "batch", {"batch": pipeline_bytes}, step_ms, None
        achieved = pipeline_bytes / (step_ms * 1e-3) / 1e9
    else:
        # roofline of the dominant kernel (largest share of device time in the
        # profiled run), its duration from the events of the timed region
        pb = pass_bytes(s)
        dom = dom_pass
        dom_ms = dom_live[dom][0] / dom_live[dom][1]
        achieved = pb[dom] / (dom_ms * 1e-3) / 1e9
        pipeline_bytes = sum(pb.values())
    variants = plan.variants(0) if not batched else {}
    if not batched:
        traffic = None if args.grid else recorded_traffic(dom, args.workload, variants.get(dom, 0))
    plain = None
    if batched:
        # the same instances one after another on one stream, no graph: the
        # plain form the batched graph call is compared with (outside the
        # timed region above)
        seq = lh.Plan(grids, autotune=not args.no_autotune)
        seq_out = torch.empty(seq.out_elems(), dtype=torch.float32, device="cuda")
        for _ in range(3):
            seq.imchi(bands, out=seq_out, mu_out=mu)
        seq.status()
        seq_steps = max(3, min(args.steps, 20))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(seq_steps):
            seq.imchi(bands, out=seq_out, mu_out=mu)
        e1.record(stream)
        torch.cuda.synchronize()
        seq.status()
        seq_ms = e0.elapsed_time(e1) / seq_steps
        # the two forms compute the same outputs
        seq.imchi(bands, out=seq_out, mu_out=mu)
        plan.imchi(bands, out=out, mu_out=mu)
        torch.cuda.synchronize()
        diff = float((seq_out - out).abs().max() / out.abs().max().clamp_min(1e-30))
        seq.close()
        del seq_out
        plain = {"ms_per_step": seq_ms, "value": outputs_per_step / world / (seq_ms * 1e-3),
                 "speedup_batched": seq_ms / step_ms, "max_rel_diff": diff}
        if persistent:
            # the earlier batched form: every instance's launches on forked
            # streams, recorded into one graph (no persistent launch)
            cg = lh.Plan(grids, graph=True, autotune=not args.no_autotune)
            cg_out = torch.empty(cg.out_elems(), dtype=torch.float32, device="cuda")
            for _ in range(3):
                cg.imchi(bands, out=cg_out, mu_out=mu)
            cg.status()
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(seq_steps):
                cg.imchi(bands, out=cg_out, mu_out=mu)
            e1.record(stream)
            torch.cuda.synchronize()
            cg.status()
            cg_ms = e0.elapsed_time(e1) / seq_steps
            plain["concurrent_graph"] = {"ms_per_step": cg_ms, "value": outputs_per_step / world / (cg_ms * 1e-3),
                                         "speedup_persistent": cg_ms / step_ms}
            cg.close()
            del cg_out
    dom_kernel = (VARIANT_KERNELS[dom][variants[dom]] if dom in VARIANT_KERNELS else KERNEL_NAMES[dom])
    tc = None
    kk = None
    thermal = None
    direct = None
    batch = None
    bwd = None
    if not batched and not args.no_tc:
        plan.imchi(bands, out=out, mu_out=mu)
        kk = kk_rpa_form(plan, out, args.steps, stream, peak)
        thermal = thermal_form(lh, grids, bands, args.steps, not args.no_autotune, stream)
        plan.imchi(bands, out=out, mu_out=mu)
        direct = energy_direct_form(lh, grids, bands, out, args.steps, mu, stream)
        bwd = backward_form(lh, grids, bands, args.steps, stream, peak, not args.no_autotune)
        try:
            batch = batched_form(lh, args.steps, not args.no_autotune, stream)
        except Exception as exc:   # an extra object: never the main line's failure
            batch = {"unavailable": str(exc)}
        tc = tensor_core_form(lh, grids, bands, out, args.steps, not args.no_autotune, mu, stream)
        if "py_inv_ms" in tc:
            tc["py_inv_ms_fp32"] = round(ptimes["py_inv"][0] / max(ptimes["py_inv"][1], 1), 5)
            tc["py_inv_roofline_frac"] = pb["py_inv"] / (tc["py_inv_ms"] * 1e-3) / 1e9 / peak

    if rank == 0:
        line = {
            "metric": "Im chi(q,w) outputs/s", "value": value, "unit": "outputs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec == lh.FP32 else "f32, p_y inverse as bf16 hi/lo products (f32 accumulation)",
            "data": "synthetic",
            "config": {"workload": args.workload,
                       "grid": f"{len(grids)} instances" if batched else f"{s.N}x{s.N} p x {s.n_eps} e",
                       "fft": "mixed" if batched else f"{s.fft_p}x{s.fft_p}x{s.fft_e}",
                       "outputs": plan.out_elems(),
                       "l2": "no flush: each step streams {:.2f} GB of intermediates through HBM, "
                             "far above the 129 MB L2".format(pipeline_bytes / 1e9),
                       "autotune": not args.no_autotune,
                       "precision": args.precision,
                       "variants": variants,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "kernel": dom_kernel, "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind,
                         "traffic": traffic, "algorithmic_bytes": pb[dom], "launch_ms": dom_ms,
                         "pipeline_frac": pipeline_bytes / (step_ms * 1e-3) / 1e9 / peak},
            "passes_ms": {k: round(v[0] / max(v[1], 1), 5) for k, v in ptimes.items()},
            "passes_note": "per-pass means from a profiled run before the timed region (events around every "
                           "pass); the timed region records events around the dominant pass only",
            "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"]},
            "e2e": {"value": e2e_value, "unit": "outputs/s", "h2d_bytes_per_step": 64 * len(grids),
                    "d2h_bytes_per_step": 4 * plan.out_elems(), "steps": e2e_steps,
                    "transfer": "each step's result to pinned host memory on a copy stream, double-buffered, "
                                "overlapped with the next step; calls replayed as CUDA graphs (graph plans)"},
            "gpu_launches": launches,
        }
        if plain is not None:
            line["plain_sequential"] = plain
        if tc is not None:
            line["tensor_core"] = tc
        if kk is not None:
            line["kk_rpa"] = kk
        if thermal is not None:
            line["finite_temperature"] = thermal
        if direct is not None:
            line["energy_direct"] = direct
        if bwd is not None:
            line["backward"] = bwd
        if batch is not None:
            line["batched_64"] = batch
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.workload)
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
