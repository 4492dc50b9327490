"""Benchmark of the randQB_b hot path on one GB300 (or N replicas under torchrun).

One step = one full randQB_b factorization (Fig. randQB_b: every block's
Omega, sketch, CholeskyQR2 with re-projection, B_i = Q_i^T A, downdate fused
with the next sketch, stop test) of the benchmark workload, with A already
resident in HBM.  Prints one JSON line.

Workloads (--workload):
  fp32  (default) 20000 x 16000 FP32, A = U diag(j^-1.5) V^T, b = 128,
        eps = 1e-2 ||A||_F, Omega seed 0 -- the plain FP32 configuration
  fp32_multiblock  the fp32 matrix at eps = 7e-4 ||A||_F (k about 1500): the
        plain FP32 path over many blocks
  fp64  2000 x 1000 FP64, s_j = 10^(-8(j-1)/999), b = 50, eps = 1e-4 ||A||_F
  mixed 32768 x 16384 FP32 on the split-TF32 tensor-core path (RQB_PREC_TF32X3),
        s_j = 10^(-4 j / 2000) for j <= 2000 then 1e-6, b = 256,
        eps = 1e-3 ||A||_F; the plain FP32 path is timed on the same matrix at
        the same eps (matched-eps comparison)
  bf16  the mixed recipe stored in BF16 (RQB_BF16: A and the residual in BF16,
        BF16 tensor-core products, Q and B in FP32), eps = 1e-2 ||A||_F; the
        plain FP32 and split-TF32 paths are timed on the same (BF16-exact)
        matrix at the same eps
  batched  512 FP32 matrices of uneven sizes, b = 32, eps_t = 1e-3 ||A_t||_F,
        one rqb_factor_batched call per step
  adjoint  8192 x 4096 FP32 (N(0,1)/sqrt(4096) plus a planted rank-64 part of
        norm 10), fixed rank k = 256, b = 64: per step the forward
        factorization, X = Q B, G = 2 (X - T) and the hand-written backward
        dL/dA of L = ||Q Q^T A - T||_F^2

The default run also measures the mixed and batched forms (a few steps each,
--no-forms skips them) and reports them under "forms" in the same line.

Metric: TFLOP/s of useful FLOPs (the algorithm's products counted once, no
extra passes of split precision):
  F = (6 s - 2) m n b + 2 m b^2 s (s - 1) + 6 m b^2 s
for s blocks of width b (sketch of block 1, per block B_i and, except for the
last block, the downdate and the next sketch; re-projection; CholeskyQR2).

--impl reference times the CPU FP64 oracle on a bounded sample of the same
workload recipe (the oracle is the reference arm: the paper has no code).
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
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "fp32": dict(name="randQB_b FP32 20000x16000 s_j=j^-1.5 b=128 eps=1e-2||A||_F", m=20000, n=16000, b=128,
                 eps_rel=1e-2, dtype="float32", spectrum="poly1.5"),
    "fp64": dict(name="randQB_b FP64 2000x1000 s_j=10^(-8(j-1)/999) b=50 eps=1e-4||A||_F", m=2000, n=1000, b=50,
                 eps_rel=1e-4, dtype="float64", spectrum="fp64cfg"),
}
WORKLOADS["fp32_multiblock"] = dict(name="randQB_b FP32 20000x16000 s_j=j^-1.5 b=128 eps=7e-4||A||_F (multi-block)",
                                    m=20000, n=16000, b=128, eps_rel=7e-4, dtype="float32", spectrum="poly1.5")
WORKLOADS["mixed"] = dict(name="randQB_b split-TF32 32768x16384 s_j=10^(-4j/2000) (j<=2000) then 1e-6 b=256 "
                               "eps=1e-3||A||_F", m=32768, n=16384, b=256, eps_rel=1e-3, dtype="float32",
                          spectrum="mixed", prec="tf32x3")
WORKLOADS["bf16"] = dict(name="randQB_b BF16 storage 32768x16384 s_j=10^(-4j/2000) (j<=2000) then 1e-6 b=256 "
                              "eps=1e-2||A||_F", m=32768, n=16384, b=256, eps_rel=1e-2, dtype="bfloat16",
                         spectrum="mixed", prec="bf16")
WORKLOADS["adjoint"] = dict(name="randQB_b fixed-rank forward + adjoint, 8192x4096 FP32, k=256, b=64", m=8192,
                            n=4096, b=64, k=256, eps_rel=0.0, dtype="float32", spectrum="adjoint")
WORKLOADS["batched"] = dict(name="randQB_b batched FP32: 512 matrices, m~U[256,4096], n~U[128,min(m,2048)], "
                                 "s_j=exp(-j/r), r~U[10,200], b=32, eps_t=1e-3||A_t||_F",
                            m=0, n=0, b=32, eps_rel=1e-3, dtype="float32", spectrum="exp", count=512)
for _k, _w in WORKLOADS.items():
    _w["key"] = _k
METRIC = "randQB_b TFLOP/s & roofline fraction at matched eps; mixed/batched vs plain FP32"


def useful_flops(m: int, n: int, b: int, s: int) -> float:
    return (6 * s - 2) * m * n * b + 2.0 * m * b * b * s * (s - 1) + 6.0 * m * b * b * s


# MMA passes of each split-TF32 product: the sketch reads Omega as exact TF32
# (hi + lo of A), the projection and the update split both operands.  On the
# split-TF32 path every product phase is one m x n x b product (the update
# is not fused with the next sketch), 2 m n b useful FLOPs per launch.
TC_PASSES = {"sketch": 2, "project": 3, "downdate": 3}
# BF16 storage: Omega and W are exact BF16 (one pass), Q_i is split (two),
# Q_i and B_i are split in the update (three).
TC_PASSES16 = {"sketch": 1, "project": 2, "downdate": 3}


def phase_flops(m: int, n: int, b: int, s: int) -> dict:
    """Algorithmic FLOPs per launch of each step of the block loop."""
    return {
        "sketch": 2.0 * m * n * b,
        "project": 2.0 * m * n * b,
        "downdate": 4.0 * m * n * b,
        "orth": (2.0 * m * b * b * s * (s - 1) + 6.0 * m * b * b * s) / max(s, 1),
    }


def spectrum(kind: str, r: int):
    import inputs
    if kind == "poly1.5":
        return inputs.spectrum_poly(r)
    if kind == "fp64cfg":
        return inputs.spectrum_fp64_config(r)
    if kind == "mixed":
        return inputs.spectrum_mixed_config(r)
    raise ValueError(kind)


def make_workload_device(w: dict, seed: int = 2):
    """A on the current CUDA device, column-major, built by inputs.usv_torch."""
    import numpy as np
    import torch
    import inputs
    m, n = w["m"], w["n"]
    s = spectrum(w["spectrum"], min(m, n))
    dt = torch.float64 if w["dtype"] == "float64" else torch.float32
    A = inputs.usv_torch(m, n, s, seed, device="cuda", dtype=dt)
    normA = float(np.sqrt(np.sum(s.astype(np.float64) ** 2)))
    if w["dtype"] == "bfloat16":
        Ab = torch.empty(n, m, dtype=torch.bfloat16, device="cuda").t()
        Ab.copy_(A)
        del A
        torch.cuda.empty_cache()
        return Ab, normA
    return A, normA


def make_sample_host(w: dict, frac: float, seed: int = 2):
    """The workload recipe at frac x the size, FP64 numpy (oracle input)."""
    import numpy as np
    import inputs
    m, n = max(8, int(w["m"] * frac)), max(8, int(w["n"] * frac))
    s = spectrum(w["spectrum"], min(m, n))
    A = inputs.usv(m, n, s, seed)
    if w["dtype"] == "float32":
        A = A.astype(np.float32).astype(np.float64)
    if w["dtype"] == "bfloat16":
        import oracle
        A = oracle.round_bf16_array(A)
    return A


class ClockSampler:
    """nvidia-smi clocks/throttle sampling in the background."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 100):
        self.gpu = gpu_index
        self.period = period_ms
        self.proc = None
        self.file = None
        self.marks = []

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", str(self.period)], stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def mark(self):
        self.marks.append(time.time())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.strip().split(",") for r in self.file.read().splitlines() if r.strip()]
        self.file.close()
        os.unlink(self.file.name)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


def alu_peak_tflops(dtype: str, num_sms: int, sm_mhz: float) -> float:
    """SIMT peak from unit counts: FP32 128 lanes/SM, FP64 2 lanes/SM (1.25 TFLOP/s
    nominal on 152 SMs at 2070 MHz), 2 FLOPs per fused multiply-add."""
    lanes = 128 if dtype == "float32" else 2
    return num_sms * lanes * 2.0 * sm_mhz * 1e6 / 1e12


# DRAM bytes (read + write) per launch of the dominant kernel, keyed by
# (workload, phase), from ncu captures (profiles/): fp32 sketch:
# k_gemm_nn_pipe at 20000 x 16000 (1.294 GB + 0.122 GB); split-TF32 and BF16
# projections and sketches: k_streamk<project|sketch> (294.9 / 283.8 MB) and
# k_streamk16<project|sketch> (148.2 / 141.8 MB) at 8192 x 8192, scaled by the
# 8x elements of a 32768 x 16384 launch (A is read once; the partials, a few
# percent, are overcounted); None where no capture of the current kernel
# exists.
NCU_TRAFFIC = {("fp32", "sketch"): 1.419e9, ("mixed", "project"): 2.359e9, ("mixed", "sketch"): 2.270e9,
               ("bf16", "project"): 1.185e9, ("bf16", "sketch"): 1.134e9}


def oracle_modes(w: dict) -> tuple[int, int]:
    """Omega precision and residual storage of the oracle run matching a workload."""
    if w["dtype"] == "float64":
        return 64, 64
    if w["dtype"] == "bfloat16":
        return 8, 16
    return 32, 64


def oracle_baseline(w: dict, frac: float, repeats: int = 1) -> dict:
    """Oracle randQB_b on the workload recipe at frac x size; TFLOP/s and cores."""
    import oracle
    A = make_sample_host(w, frac)
    m, n = A.shape
    nA = float((A * A).sum()) ** 0.5
    eps = w["eps_rel"] * nA
    prec, store = oracle_modes(w)
    times = []
    res = None
    for _ in range(repeats):
        t0 = time.perf_counter()
        res = oracle.randqb_b(A, eps, w["b"], seed=0, omega_prec=prec, storage_prec=store)
        times.append(time.perf_counter() - t0)
    t = statistics.median(times)
    F = useful_flops(m, n, w["b"], res.blocks)
    return {"value": F / t / 1e12, "unit": "TFLOP/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"oracle randQB_b on the same recipe at {m}x{n} (frac {frac}), b={w['b']}, "
                      f"eps={w['eps_rel']}||A||_F, k={res.k}, {t:.2f} s per run", "seconds": t}


def run_ours(args, w: dict, rank: int, world: int, dist):
    import torch
    from paper_1503_07157_gb300 import build as _build
    _build.build()
    from paper_1503_07157_gb300 import rqb

    dev = torch.device("cuda", torch.cuda.current_device())
    A, normA = make_workload_device(w)
    m, n, b = w["m"], w["n"], w["b"]
    eps = w["eps_rel"] * normA
    dt = {"float64": torch.float64, "float32": torch.float32, "bfloat16": torch.bfloat16}[w["dtype"]]
    prec = {"tf32x3": rqb.RQB_PREC_TF32X3, "bf16": rqb.RQB_PREC_BF16}.get(w.get("prec"), rqb.RQB_PREC_NATIVE)
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    h = rqb.Handle(dt, prec=prec, stream=stream, flags=rqb.RQB_FLAG_PHASE_TIMING)
    for _ in range(args.warmup):
        _, _, k, rc = h.rqb_factor(A, eps, b, seed=0)
    st = h.rqb_get_stats()
    s_blocks, k = st.blocks, st.k

    def barrier():
        if dist is not None:
            dist.barrier()

    phase_ms = [0.0] * rqb.RQB_NUM_PHASES
    phase_calls = [0] * rqb.RQB_NUM_PHASES
    launches = 0
    clocks = ClockSampler(torch.cuda.current_device())
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.start()
    time.sleep(0.25)
    ev0.record(stream)
    for _ in range(args.steps):
        _, _, kk, rc = h.rqb_factor(A, eps, b, seed=0)
        stt = h.rqb_get_stats()
        for i in range(rqb.RQB_NUM_PHASES):
            phase_ms[i] += stt.phase_ms[i]
            phase_calls[i] += stt.phase_calls[i]
        launches += stt.kernel_launches
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, dist, dev)
    F = useful_flops(m, n, b, s_blocks)
    value = aggregate_value(F, world, ms)

    # roofline of the dominant product step (its main kernel plus split reduction)
    pf = phase_flops(m, n, b, s_blocks)
    names = list(rqb.PHASES)
    per_step = {names[i]: round(phase_ms[i] / args.steps, 4) for i in range(len(names))}
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    props = torch.cuda.get_device_properties(dev)
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    es = {"float32": 4, "float64": 8, "bfloat16": 2}[w["dtype"]]
    if prec in (rqb.RQB_PREC_TF32X3, rqb.RQB_PREC_BF16):
        is16 = prec == rqb.RQB_PREC_BF16
        table = TC_PASSES16 if is16 else TC_PASSES
        cand = [(phase_ms[i], names[i]) for i in range(len(names)) if names[i] in table and phase_calls[i] > 0]
        dom_ms, dom = max(cand)
        idx = names.index(dom)
        per_launch_ms = phase_ms[idx] / phase_calls[idx]
        passes = table[dom]
        # useful work of one launch (each product phase is one m x n x b product
        # on the tensor-core path), its algorithmic bytes (one read of A; the
        # update also writes it), and the roofline time on those terms: split
        # passes are work the kernel executes, not useful work
        useful = 2.0 * m * n * b
        nbytes = (2 if dom == "downdate" else 1) * m * n * es
        t = per_launch_ms * 1e-3
        bf16 = float(peaks.get("bf16_tflops", 1900.0))
        peak_tc = bf16 if is16 else bf16 / 2.0
        t_tc, t_hbm = useful / (peak_tc * 1e12), nbytes / (hbm * 1e9)
        sfx = "16" if is16 else ""
        kern = {"sketch": f"k_streamk{sfx}<sketch> + k_reduce_sketch",
                "project": f"k_streamk{sfx}<project> + k_reduce_project{sfx}",
                "downdate": f"k_update{sfx}w" if n >= 256 else f"k_update{sfx}"}[dom]
        tc_src = (f"measured bf16 burst {bf16} TFLOP/s (MEASURED_PEAKS.json), of measured" if is16
                  else f"measured bf16 burst {bf16} TFLOP/s (MEASURED_PEAKS.json) x 1/2 (nominal TF32:BF16 dense "
                       f"ratio), of measured")
        if t_hbm >= t_tc:
            roofline = {"bound": "hbm", "kernel": kern, "achieved": round(nbytes / t / 1e9, 1), "peak": hbm,
                        "unit": "GB/s", "frac": round(t_hbm / t, 4),
                        "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs), of measured"}
        else:
            roofline = {"bound": "tensor", "kernel": kern, "achieved": round(useful / t / 1e12, 3),
                        "peak": round(peak_tc, 3), "unit": "TFLOP/s", "frac": round(t_tc / t, 4),
                        "peak_source": tc_src}
        roofline.update({"traffic": NCU_TRAFFIC.get((w.get("key"), dom)),
                         "bytes_per_launch": nbytes, "useful_flops_per_launch": useful,
                         "roof_ms": round(max(t_tc, t_hbm) * 1e3, 4), "launch_ms": round(per_launch_ms, 4),
                         "useful_tflops": round(useful / t / 1e12, 3), "hbm_gbs": round(nbytes / t / 1e9, 1),
                         "mma_passes": passes, "executed_tflops": round(passes * useful / t / 1e12, 3),
                         "executed_frac": round(passes * useful / t / 1e12 / peak_tc, 4),
                         "tensor_peak": round(peak_tc, 3), "tensor_peak_source": tc_src,
                         "phase_ms_per_step": per_step})
        peak_run = peak_tc
        peak_run_src = tc_src
    else:
        cand = [(phase_ms[i], names[i]) for i in range(len(names)) if names[i] in pf and phase_calls[i] > 0]
        dom_ms, dom = max(cand)
        idx = names.index(dom)
        per_launch_ms = phase_ms[idx] / phase_calls[idx]
        achieved = pf[dom] / (per_launch_ms * 1e-3) / 1e12
        peak = alu_peak_tflops(w["dtype"], props.multi_processor_count, sm_max)
        roofline = {"bound": "alu",
                    "kernel": f"{dom} (k_gemm_{'nn_pipe' if dom == 'sketch' else 'tn'} + split reduction)"
                    if dom in ("sketch", "project") else dom,
                    "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "TFLOP/s",
                    "frac": round(achieved / peak, 4), "traffic": NCU_TRAFFIC.get((w.get("key"), dom)),
                    "peak_source": f"derived: {props.multi_processor_count} SMs x "
                                   f"{'128 FP32' if w['dtype'] == 'float32' else '2 FP64'} lanes x 2 x {sm_max:.0f} MHz",
                    "phase_ms_per_step": per_step}
        peak_run, peak_run_src = peak, roofline["peak_source"]
    whole = whole_run_roofline(F, m, n, s_blocks, es, ms, peak_run, peak_run_src, hbm)
    return dict(h=h, A=A, eps=eps, value=value, ms=ms, F=F, k=k, s=s_blocks, clocks=clk, roofline=roofline,
                whole_run=whole, launches=launches // max(args.steps, 1), stream=stream)


def whole_run_roofline(F: float, m: int, n: int, s: int, es: int, ms: float, peak_tflops: float, peak_src: str,
                       hbm_gbs: float) -> dict:
    """Roofline of one whole factorization: the useful FLOPs F at the path's
    arithmetic peak against the algorithmic bytes Bt = (3s - 1) m n sizeof(A)
    (A read by the first sketch, then per non-last block one read for B_i and
    one read + write for the downdate fused with the next sketch, then one read
    for the last B_i) at the measured HBM bandwidth; frac = roofline time /
    measured time."""
    Bt = (3 * s - 1) * m * n * es
    t_f, t_b = F / (peak_tflops * 1e12), Bt / (hbm_gbs * 1e9)
    return {"useful_flops": F, "bytes": Bt, "flop_ms": round(t_f * 1e3, 4), "byte_ms": round(t_b * 1e3, 4),
            "bound": "hbm" if t_b >= t_f else "compute", "roof_ms": round(max(t_f, t_b) * 1e3, 4),
            "measured_ms": round(ms, 4), "frac": round(max(t_f, t_b) * 1e3 / ms, 4),
            "peak_tflops": round(peak_tflops, 3), "peak_source": peak_src, "hbm_gbs": hbm_gbs}


def adjoint_flops(m: int, n: int, k: int) -> float:
    """Useful FLOPs of rqb_backward: R = B Omega, Q^T G, Q (Q^T G), G B^T,
    G^T Q, A (G^T Q), Q^T M, Q (Q^T M), M R^-T, N Omega^T."""
    return 12.0 * m * n * k + 6.0 * m * k * k + 2.0 * n * k * k


def run_adjoint(args, w: dict, rank: int, world: int, dist) -> dict:
    """Config-5 workload: forward at fixed rank, X = Q B, G = 2 (X - T), backward."""
    import torch
    import inputs
    from paper_1503_07157_gb300 import build as _build
    _build.build()
    from paper_1503_07157_gb300 import rqb
    m, n, b, k = w["m"], w["n"], w["b"], w["k"]
    A_np, T_np, _ = inputs.config_adjoint_np(m=m, n=n, seed=5, rank=64, norm=10.0)
    A = torch.as_tensor(A_np.T, dtype=torch.float32, device="cuda").t()
    T = torch.as_tensor(T_np.T, dtype=torch.float32, device="cuda").t()
    del A_np, T_np
    stream = torch.cuda.Stream()
    h = rqb.Handle(torch.float32, stream=stream, max_rank=k, fixed_rank=True)

    def step():
        h.rqb_factor(A, 0.0, b, seed=0)
        X = h.rqb_reconstruct(m, n)
        with torch.cuda.stream(stream):
            G = 2.0 * (X - T)
        return h.rqb_backward(G)

    for _ in range(args.warmup):
        step()
    clocks = ClockSampler(torch.cuda.current_device())
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.25)
    launches = 0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
        launches += h.rqb_get_stats().kernel_launches
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, dist, torch.device("cuda", torch.cuda.current_device()))
    s_blocks = k // b
    F = useful_flops(m, n, b, s_blocks) + 2.0 * m * n * k + adjoint_flops(m, n, k)   # forward, X = Q B, backward
    h.close()
    peaks = measured_peaks()
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    peak = alu_peak_tflops("float32", props.multi_processor_count, float(peaks.get("sm_max_mhz", 2070.0)))
    value = aggregate_value(F, world, ms)
    return dict(value=value, ms=ms, F=F, clocks=clk, launches=launches // max(args.steps, 1),
                roofline={"bound": "alu", "kernel": "whole step (SIMT GEMMs of forward and backward)",
                          "achieved": round(F / (ms * 1e-3) / 1e12, 3), "peak": round(peak, 3), "unit": "TFLOP/s",
                          "frac": round(F / (ms * 1e-3) / 1e12 / peak, 4), "traffic": None,
                          "peak_source": f"derived: {props.multi_processor_count} SMs x 128 FP32 lanes x 2 x "
                                         f"{float(peaks.get('sm_max_mhz', 2070.0)):.0f} MHz"})


def run_plain_matched(args, w: dict, res: dict, steps: int = 2, prec: int | None = None) -> dict:
    """The plain FP32 path (RQB_PREC_NATIVE; or the split-TF32 path with prec)
    on the same matrix (widened to FP32 for a BF16 workload) at the same eps."""
    import torch
    from paper_1503_07157_gb300 import rqb
    m, n, b = w["m"], w["n"], w["b"]
    prec = rqb.RQB_PREC_NATIVE if prec is None else prec
    A = res["A"]
    if A.dtype != torch.float32:
        A32 = torch.empty(n, m, dtype=torch.float32, device=A.device).t()
        A32.copy_(A)
        A = A32
    h = rqb.Handle(torch.float32, prec=prec, stream=res["stream"])
    _, _, k, rc = h.rqb_factor(A, res["eps"], b, seed=0)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(res["stream"])
    for _ in range(steps):
        _, _, k, rc = h.rqb_factor(A, res["eps"], b, seed=0)
    ev1.record(res["stream"])
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    s_blocks = h.rqb_get_stats().blocks
    h.close()
    del A
    F = useful_flops(m, n, b, s_blocks)
    name = "split-TF32 (RQB_PREC_TF32X3)" if prec == rqb.RQB_PREC_TF32X3 else "plain FP32 (RQB_PREC_NATIVE)"
    return {"impl": name, "ms_per_step": round(ms, 3), "value": round(F / (ms * 1e-3) / 1e12, 4),
            "unit": "TFLOP/s", "k": k, "steps": steps, "speedup_of_form": round(ms / res["ms"], 3)}


def run_omega_smem(args, w: dict, res: dict, steps: int = 3) -> dict:
    """The BF16 workload with Omega_i drawn inside the sketch kernel
    (RQB_FLAG_OMEGA_SMEM) instead of loaded from its buffer: same matrix, eps
    and results; the sketch phase and the whole factorization timed."""
    import torch
    from paper_1503_07157_gb300 import rqb
    m, n, b = w["m"], w["n"], w["b"]
    h = rqb.Handle(torch.bfloat16, prec=rqb.RQB_PREC_BF16, stream=res["stream"],
                   flags=rqb.RQB_FLAG_PHASE_TIMING | rqb.RQB_FLAG_OMEGA_SMEM)
    h.rqb_factor(res["A"], res["eps"], b, seed=0)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sk_ms, sk_calls = 0.0, 0
    torch.cuda.synchronize()
    ev0.record(res["stream"])
    for _ in range(steps):
        _, _, k, rc = h.rqb_factor(res["A"], res["eps"], b, seed=0)
        st = h.rqb_get_stats()
        sk_ms += st.phase_ms[0]
        sk_calls += st.phase_calls[0]
    ev1.record(res["stream"])
    torch.cuda.synchronize()
    h.close()
    ms = ev0.elapsed_time(ev1) / steps
    buf = res["roofline"]["phase_ms_per_step"]["sketch"]
    return {"impl": "BF16, Omega_i drawn in shared memory inside the sketch (RQB_FLAG_OMEGA_SMEM)",
            "ms_per_step": round(ms, 3), "k": k, "steps": steps,
            "sketch_ms_per_step": round(sk_ms / steps, 4), "sketch_ms_per_launch": round(sk_ms / max(sk_calls, 1), 4),
            "buffered_sketch_ms_per_step": buf, "buffered_ms_per_step": round(res["ms"], 3)}


def run_e2e(args, w: dict, res: dict) -> dict:
    """Same metric through rqb_factor_host: pinned host A in, Q and B back to
    pinned host buffers, all copies inside the timed region."""
    import torch
    from paper_1503_07157_gb300 import rqb
    m, n, b = w["m"], w["n"], w["b"]
    dt = res["A"].dtype
    dto = torch.float64 if dt == torch.float64 else torch.float32
    cap = min(m, n, args.e2e_max_rank)
    A_host = torch.empty(n, m, dtype=dt, pin_memory=True).t()
    A_host.copy_(res["A"])
    Q_host = torch.empty(cap, m, dtype=dto, pin_memory=True).t()
    B_host = torch.empty(n, cap, dtype=dto, pin_memory=True).t()
    prec = {"tf32x3": rqb.RQB_PREC_TF32X3, "bf16": rqb.RQB_PREC_BF16}.get(w.get("prec"), rqb.RQB_PREC_NATIVE)
    h = rqb.Handle(dt, prec=prec, stream=res["stream"], max_rank=cap)
    times, k = [], 0
    for i in range(args.warmup + max(1, args.e2e_steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        k, rc = h.rqb_factor_host(A_host, res["eps"], b, 0, Q_host, B_host)
        t1 = time.perf_counter()
        if i >= args.warmup:
            times.append(t1 - t0)
    h.close()
    t = statistics.median(times)
    es, eo = A_host.element_size(), Q_host.element_size()
    return {"value": round(res["F"] / t / 1e12, 4), "unit": "TFLOP/s", "h2d_bytes_per_step": m * n * es,
            "d2h_bytes_per_step": (m * k + k * n) * eo, "ms_per_step": round(t * 1e3, 3),
            "api": "rqb_factor_host (pinned host buffers)"}


def make_batch_device(count: int, seed: int = 0):
    import inputs
    return inputs.config_batched_torch(count, seed=seed)


def run_batched(args, w: dict, rank: int, world: int, dist, do_e2e: bool = True):
    """Config-4 workload: one rqb_factor_batched call per step."""
    import torch
    from paper_1503_07157_gb300 import build as _build
    _build.build()
    from paper_1503_07157_gb300 import rqb
    mats, eps, cases = make_batch_device(w["count"])
    b = w["b"]
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    h = rqb.Handle(torch.float32, stream=stream)
    for _ in range(args.warmup):
        out = h.rqb_factor_batched(mats, eps, b, seed=0)
    ks = [o[2] for o in out]
    sts = [o[3] for o in out]
    F = sum(useful_flops(c.m, c.n, b, (k + b - 1) // b) for c, k in zip(cases, ks))
    clocks = ClockSampler(torch.cuda.current_device())
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.25)
    kern_ms = 0.0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    launches = 0
    for _ in range(args.steps):
        h.rqb_factor_batched(mats, eps, b, seed=0)
        stb = h.rqb_get_stats()
        kern_ms += stb.phase_ms[0]
        launches += stb.kernel_launches
    tile_width = stb.tile_width
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, dist, torch.device("cuda", torch.cuda.current_device()))
    kern_ms /= args.steps
    peaks = measured_peaks()
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    peak = alu_peak_tflops("float32", props.multi_processor_count, float(peaks.get("sm_max_mhz", 2070.0)))
    achieved = F / (kern_ms * 1e-3) / 1e12
    # the same matrices through a loop of single-matrix rqb_factor calls (one pass)
    h1 = rqb.Handle(torch.float32, stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for A, e in zip(mats, eps):
        h1.rqb_factor(A, e, b, 0, check=False)
    torch.cuda.synchronize()
    loop_ms = (time.perf_counter() - t0) * 1e3
    h1.close()
    # the byte model of the schedule, beside the ALU bound: per matrix of s
    # blocks, A crosses HBM (3 s - 1) times (first sketch, each projection,
    # each update read + write) and block i reads Qbar (i - 1) b columns twice
    # for the re-projection
    model_bytes = 0.0
    for c, k in zip(cases, ks):
        sb = (k + b - 1) // b
        model_bytes += 4.0 * ((3 * sb - 1) * c.m * c.n + 2.0 * c.m * b * sb * (sb - 1) / 2.0)
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    hbm_gbs = model_bytes / (ms * 1e-3) / 1e9
    roofline = {"bound": "alu", "kernel": "grouped batched kernels (k_rows_update, k_cols, k_rows, k_mat), whole batch "
                          f"as one graph launch, projection tile width {tile_width} (autotuned)",
                "achieved": round(achieved, 3),
                "peak": round(peak, 3), "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": None,
                "peak_source": f"derived: {props.multi_processor_count} SMs x 128 FP32 lanes x 2 x "
                               f"{float(peaks.get('sm_max_mhz', 2070.0)):.0f} MHz",
                "byte_model": {"bytes_per_step": model_bytes, "achieved_gbs": round(hbm_gbs, 1),
                               "peak_gbs": hbm_peak, "frac": round(hbm_gbs / hbm_peak, 4),
                               "note": "(3s-1) crossings of each A plus the re-projection reads; "
                                       "the ALU bound is the binding one (16 flop/B > ridge)"}}
    t_f, t_b = F / (peak * 1e12), model_bytes / (hbm_peak * 1e9)
    whole = {"useful_flops": F, "bytes": model_bytes, "flop_ms": round(t_f * 1e3, 4), "byte_ms": round(t_b * 1e3, 4),
             "bound": "hbm" if t_b >= t_f else "compute", "roof_ms": round(max(t_f, t_b) * 1e3, 4),
             "measured_ms": round(ms, 4), "frac": round(max(t_f, t_b) * 1e3 / ms, 4), "peak_tflops": round(peak, 3),
             "peak_source": roofline["peak_source"], "hbm_gbs": hbm_peak}
    if not do_e2e:
        h.close()
        return dict(value=aggregate_value(F, world, ms), ms=ms, F=F, clocks=clk, roofline=roofline, e2e=None,
                    whole_run=whole,
                    launches=launches // max(args.steps, 1), extra={"count": len(mats), "k_mean": float(sum(ks)) / len(ks), "k_max": max(ks),
                                       "projection_tile_width": tile_width,
                                       "status_ok": int(sum(1 for s_ in sts if s_ == 0)),
                                       "loop_of_single_calls_ms": round(loop_ms, 2)})
    # e2e: pinned host inputs in, Q and B back to pinned host, inside the timed region
    hosts = [torch.empty(A.shape[1], A.shape[0], dtype=torch.float32, pin_memory=True).t() for A in mats]
    for hA, A in zip(hosts, mats):
        hA.copy_(A)
    dev = [torch.empty_like(A).t().contiguous().t() for A in mats]
    e2e_times = []
    h2d = sum(A.numel() * 4 for A in mats)
    d2h = 0
    for it in range(args.warmup + max(1, args.e2e_steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for d_, hA in zip(dev, hosts):
                d_.copy_(hA, non_blocking=True)
        out2 = h.rqb_factor_batched(dev, eps, b, seed=0)
        with torch.cuda.stream(stream):
            qb = [(Q.to("cpu", non_blocking=True), B.to("cpu", non_blocking=True)) for Q, B, _, _ in out2]
        stream.synchronize()
        t1 = time.perf_counter()
        if it >= args.warmup:
            e2e_times.append(t1 - t0)
            d2h = sum(q.numel() * 4 + bb.numel() * 4 for q, bb in qb)
    te = statistics.median(e2e_times)
    e2e = {"value": round(F / te / 1e12, 4), "unit": "TFLOP/s", "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(d2h), "ms_per_step": round(te * 1e3, 3),
           "api": "pinned host copies + rqb_factor_batched"}
    h.close()
    return dict(value=aggregate_value(F, world, ms), ms=ms, F=F, clocks=clk, roofline=roofline, e2e=e2e,
                whole_run=whole,
                launches=launches // max(args.steps, 1), extra={"count": len(mats), "k_mean": float(sum(ks)) / len(ks), "k_max": max(ks),
                                   "projection_tile_width": tile_width,
                                   "status_ok": int(sum(1 for s_ in sts if s_ == 0)),
                                   "loop_of_single_calls_ms": round(loop_ms, 2)})


def max_over_ranks(ms: float, dist, device=None) -> float:
    """The slowest replica's time: the maximum of a per-rank value over all ranks."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(flops_per_rank: float, world: int, ms: float) -> float:
    """Whole-job TFLOP/s: the work of all replicas over the slowest replica's time."""
    return flops_per_rank * world / (ms * 1e-3) / 1e12


def init_dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world <= 1:
        return 0, 1, None
    import torch
    import torch.distributed as dist
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist.init_process_group("nccl")
    return rank, world, dist


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="fp32")
    ap.add_argument("--sample-frac", type=float, default=0.3,
                    help="size fraction of the oracle's bounded sample (CPU baseline / reference arm)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--e2e-max-rank", type=int, default=4096)
    ap.add_argument("--no-forms", action="store_true",
                    help="default workload only: skip the mixed and batched forms")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    w = WORKLOADS[args.workload]

    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        if rank != 0:
            return 0
        return run_reference(args, w)

    import torch
    rank, world, dist = init_dist()
    if args.workload == "batched":
        return main_batched(args, w, rank, world, dist)
    if args.workload == "adjoint":
        r = run_adjoint(args, w, rank, world, dist)
        if rank == 0:
            line = {"metric": METRIC, "value": round(r["value"], 4), "unit": "TFLOP/s", "n_gpus": world,
                    "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(r["ms"], 3),
                    "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                    "data": "synthetic (N(0,1)/sqrt(n) plus a planted rank-64 part; T ~ N(0,1))",
                    "config": {"workload": w["name"], "m": w["m"], "n": w["n"], "b": w["b"], "k": w["k"],
                               "useful_flops_per_step": r["F"], "parallelism": f"replicas x{world}" if world > 1
                               else "single GPU", "l2": "inputs larger than L2 (A is 0.13 GB, T and G too)"},
                    "roofline": r["roofline"], "cpu_baseline": None, "e2e": None,
                    "gpu_launches": r["launches"] * args.steps, "clocks": r["clocks"]}
            print(json.dumps(line), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return 0
    res = run_ours(args, w, rank, world, dist)
    e2e = run_e2e(args, w, res) if rank == 0 else None
    matched = run_plain_matched(args, w, res) if (rank == 0 and w.get("prec") in ("tf32x3", "bf16")) else None
    matched_tc = None
    if rank == 0 and w.get("prec") == "bf16":
        from paper_1503_07157_gb300 import rqb as _rqb
        matched_tc = run_plain_matched(args, w, res, prec=_rqb.RQB_PREC_TF32X3)
    forms = None
    if args.workload == "fp32" and not args.no_forms:
        forms = run_forms(args, rank, world, dist)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_baseline(w, args.sample_frac)
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(res["value"], 4), "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(res["ms"], 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"float32": "f32", "float64": "f64", "bfloat16": "bf16 (A, W; FP32 accumulate, FP32 Q/B)"}[
                w["dtype"]], "data": "synthetic (seeded A = U diag(s) V^T, U, V from QR of "
            "Gaussian matrices; Omega Philox4x32-10 + Box-Muller)",
            "config": {"workload": w["name"], "m": w["m"], "n": w["n"], "b": w["b"], "eps_rel": w["eps_rel"],
                       "k": res["k"], "blocks": res["s"], "useful_flops_per_step": res["F"],
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "input larger than L2 (A is %.2f GB)" % (w["m"] * w["n"] *
                                                                       {"float32": 4, "float64": 8, "bfloat16": 2}[
                                                                           w["dtype"]] / 1e9)
                       if w["m"] * w["n"] * 4 > 129e6 else "L2 not flushed: input fits in L2"},
            "roofline": res["roofline"], "whole_run": res["whole_run"], "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": res["launches"]
            * args.steps, "clocks": res["clocks"],
        }
        if matched is not None:
            line["plain_fp32_matched_eps"] = matched
        if matched_tc is not None:
            line["split_tf32_matched_eps"] = matched_tc
        if forms is not None:
            line["forms"] = forms
        if cpu is not None:
            cpu.pop("seconds", None)
        print(json.dumps(line), flush=True)
    res["h"].close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_forms(args, rank: int, world: int, dist) -> dict:
    """The mixed (split-TF32) and batched forms, a few steps each, for the
    default line: value, ms, roofline, and the plain FP32 comparison."""
    import copy
    import gc
    import torch
    out = {}
    a = copy.copy(args)
    a.steps, a.warmup = 3, 3
    # the plain FP32 path over many blocks (re-projection, fused downdate and
    # next sketch) on the default workload's matrix
    wf = WORKLOADS["fp32_multiblock"]
    r = run_ours(a, wf, rank, world, dist)
    out["fp32_multiblock"] = {"workload": wf["name"], "value": round(r["value"], 4), "unit": "TFLOP/s",
                              "ms_per_step": round(r["ms"], 3), "steps": a.steps, "k": r["k"], "blocks": r["s"],
                              "roofline": r["roofline"], "whole_run": r["whole_run"]}
    r["h"].close()
    del r
    gc.collect()
    torch.cuda.empty_cache()
    # the FP64 path (2000 x 1000, b = 50, twelve blocks; A fits in L2)
    wd = WORKLOADS["fp64"]
    a.steps = 10
    r = run_ours(a, wd, rank, world, dist)
    out["fp64"] = {"workload": wd["name"], "value": round(r["value"], 4), "unit": "TFLOP/s",
                   "ms_per_step": round(r["ms"], 3), "steps": a.steps, "k": r["k"], "blocks": r["s"],
                   "roofline": r["roofline"], "whole_run": r["whole_run"],
                   "l2": "input fits in L2 (16 MB) and is not flushed"}
    r["h"].close()
    del r
    gc.collect()
    torch.cuda.empty_cache()
    a.steps = 5
    wm = WORKLOADS["mixed"]
    r = run_ours(a, wm, rank, world, dist)
    out["mixed"] = {"workload": wm["name"], "value": round(r["value"], 4), "unit": "TFLOP/s",
                    "ms_per_step": round(r["ms"], 3), "steps": a.steps, "k": r["k"], "blocks": r["s"],
                    "roofline": r["roofline"], "whole_run": r["whole_run"],
                    "plain_fp32_matched_eps": run_plain_matched(a, wm, r) if rank == 0 else None}
    r["h"].close()
    del r
    gc.collect()
    torch.cuda.empty_cache()
    w16 = WORKLOADS["bf16"]
    r = run_ours(a, w16, rank, world, dist)
    out["bf16"] = {"workload": w16["name"], "value": round(r["value"], 4), "unit": "TFLOP/s",
                   "ms_per_step": round(r["ms"], 3), "steps": a.steps, "k": r["k"], "blocks": r["s"],
                   "roofline": r["roofline"], "whole_run": r["whole_run"],
                   "plain_fp32_matched_eps": run_plain_matched(a, w16, r) if rank == 0 else None,
                   "omega_in_shared_memory": run_omega_smem(a, w16, r) if rank == 0 else None}
    r["h"].close()
    del r
    gc.collect()
    torch.cuda.empty_cache()
    wb = WORKLOADS["batched"]
    a.steps = 2
    rb = run_batched(a, wb, rank, world, dist, do_e2e=False)
    out["batched"] = dict({"workload": wb["name"], "value": round(rb["value"], 4), "unit": "TFLOP/s",
                           "ms_per_step": round(rb["ms"], 3), "steps": a.steps, "roofline": rb["roofline"],
                           "whole_run": rb["whole_run"]},
                          **rb["extra"])
    out["batched"]["speedup_vs_loop_of_single_calls"] = round(rb["extra"]["loop_of_single_calls_ms"] / rb["ms"], 3)
    gc.collect()
    torch.cuda.empty_cache()
    wa = WORKLOADS["adjoint"]
    a.steps = 10
    ra = run_adjoint(a, wa, rank, world, dist)
    out["adjoint"] = {"workload": wa["name"], "value": round(ra["value"], 4), "unit": "TFLOP/s",
                      "ms_per_step": round(ra["ms"], 3), "steps": a.steps, "roofline": ra["roofline"]}
    return out


def main_batched(args, w, rank, world, dist) -> int:
    res = run_batched(args, w, rank, world, dist)
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = oracle_baseline_batched(w, args.sample_frac)
        line = {"metric": METRIC, "value": round(res["value"], 4), "unit": "TFLOP/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(res["ms"], 3),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic (seeded A_t = U diag(s) V^T; sizes drawn from seed 0)",
                "config": dict({"workload": w["name"], "b": w["b"], "eps_rel": w["eps_rel"],
                                "useful_flops_per_step": res["F"],
                                "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                                "l2": "inputs larger than L2 (4.9 GB in total)"}, **res["extra"]),
                "roofline": res["roofline"], "whole_run": res["whole_run"], "cpu_baseline": cpu, "e2e": res["e2e"],
                "gpu_launches": res["launches"] * args.steps, "clocks": res["clocks"]}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def oracle_baseline_batched(w: dict, frac: float) -> dict:
    """Oracle on the first matrices of the batch recipe (bounded sample)."""
    import numpy as np
    import oracle
    import inputs
    cases = inputs.batched_sizes(w["count"], seed=0)
    t_tot, F = 0.0, 0.0
    used = 0
    for i, c in enumerate(cases):
        if t_tot > 10.0:
            break
        A = inputs.usv(c.m, c.n, inputs.spectrum_exp(min(c.m, c.n), c.rate), 1000 + i).astype(np.float32).astype(np.float64)
        eps = 1e-3 * float(np.linalg.norm(A))
        t0 = time.perf_counter()
        r = oracle.randqb_b(A, eps, w["b"], seed=0, omega_prec=32)
        t_tot += time.perf_counter() - t0
        F += useful_flops(c.m, c.n, w["b"], r.blocks)
        used += 1
    return {"value": F / t_tot / 1e12, "unit": "TFLOP/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"oracle randQB_b on the first {used} matrices of the batch recipe ({t_tot:.1f} s)"}


def run_reference(args, w: dict) -> int:
    """The reference arm: the CPU FP64 oracle, as it stands, on the machine's host
    cores; each step is one run on the bounded sample of the workload recipe."""
    import oracle
    if args.workload == "batched":
        cb = oracle_baseline_batched(w, args.sample_frac)
        line = {"impl": "reference", "metric": METRIC, "value": round(cb["value"], 6), "unit": "TFLOP/s",
                "n_gpus": 0, "steps": 1, "warmup": 0, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": {"workload": w["name"]},
                "cpu_baseline": cb, "e2e": {"value": round(cb["value"], 6), "unit": "TFLOP/s",
                                            "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0
    # exactly W untimed and K timed runs; the sample is shrunk (from one
    # calibration run) so that they take about REF_BUDGET_S on the host cores
    REF_BUDGET_S = 150.0
    steps, warm = max(1, args.steps), max(0, args.warmup)
    prec, store = oracle_modes(w)
    frac = args.sample_frac

    def sample(f):
        A = make_sample_host(w, f)
        return A, w["eps_rel"] * float((A * A).sum()) ** 0.5

    A, eps = sample(frac)
    t0 = time.perf_counter()
    oracle.randqb_b(A, eps, w["b"], seed=0, omega_prec=prec, storage_prec=store)
    t_cal = time.perf_counter() - t0
    if (warm + steps) * t_cal > REF_BUDGET_S:
        # time grows with m n at a fixed rank: frac scales by the square root
        frac = max(0.05, frac * ((REF_BUDGET_S / ((warm + steps) * t_cal)) ** 0.5))
        A, eps = sample(frac)
    m, n = A.shape
    times, r = [], None
    for i in range(warm + steps):
        t0 = time.perf_counter()
        r = oracle.randqb_b(A, eps, w["b"], seed=0, omega_prec=prec, storage_prec=store)
        if i >= warm:
            times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    F = useful_flops(m, n, w["b"], r.blocks)
    val = F / t / 1e12
    line = {"impl": "reference", "metric": METRIC, "value": round(val, 6), "unit": "TFLOP/s", "n_gpus": 0,
            "steps": steps, "warmup": warm, "ms_per_step": round(t * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["name"], "sample": f"{m}x{n}", "k": r.k, "blocks": r.blocks},
            "cpu_baseline": {"value": round(val, 6), "unit": "TFLOP/s", "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": f"same recipe at {m}x{n} (frac {frac:.3f}, sized so that "
                             f"{warm} warm-up and {steps} timed runs take about {REF_BUDGET_S:.0f} s)"},
            "e2e": {"value": round(val, 6), "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
