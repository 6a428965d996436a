#!/usr/bin/env python
"""Benchmark of the projected-gradient deconvolution hot path.

Workload (default ``ring3d``): X 512x512x128 filaments, H 31x31x21
Gaussian-plus-ring template, Y = X (*) H with Poisson noise.  One step is one
accepted iteration of Steps 1-3: the adjoint convolution with the projected
update, the forward convolution with the residual, and the FP64 decision on
the device.  The timed region is one ``cdv_iterate`` call of K steps (a CUDA
graph replay; it also runs the initial forward convolution of x_0).

Metric: GMAC/s = algorithmic multiply-adds (convolutions executed x
prod(m) x prod(2p+1)) / device time; iterations/s is reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cdv|reference]
Under torchrun each rank solves its own copy of the workload (weak scaling);
rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
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

SM_COUNT = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0
FP32_PEAK_TFLOPS = SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12   # 80.55

def measured_peaks():
    """Measured BF16 dense peak of this machine's GPUs (TFLOP/s), else the recipe's fallback."""
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def measured_hbm():
    """Measured HBM copy bandwidth of this machine's GPUs (GB/s), else the recipe's fallback."""
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# Peaks measured in this process on the GPU (filled by measure_peaks): the library's FP32 FMA probe and a
# cuBLAS TF32 GEMM burst.
LIVE_PEAKS = {}


def measure_peaks(stream):
    """FP32 FMA rate (cdv_probe_fp32_fma, CUDA events, best of 3) and the TF32 dense GEMM burst rate
    (torch.matmul on float32 with TF32 allowed, 8192^3, best of 5), in TFLOP/s."""
    import ctypes

    import torch

    from paper_1711_11224_gb300 import _binding
    lib = _binding.load()
    blocks, threads, iters = SM_COUNT * 4, 512, 1 << 15
    out = torch.empty(blocks * threads, device="cuda", dtype=torch.float32)
    best = None
    for _ in range(4):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _binding.check(lib.cdv_probe_fp32_fma(ctypes.c_void_p(out.data_ptr()), blocks, threads, iters,
                                              ctypes.c_void_p(stream.cuda_stream)))
        b.record(stream)
        b.synchronize()
        t = a.elapsed_time(b) / 1e3
        best = t if best is None else min(best, t)
    LIVE_PEAKS["fp32_ffma"] = 16.0 * iters * blocks * threads / best / 1e12
    n = 8192
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        A = torch.randn(n, n, device="cuda")
        B = torch.randn(n, n, device="cuda")
        C = torch.empty(n, n, device="cuda")
        torch.matmul(A, B, out=C)
        torch.cuda.synchronize()
        best = None
        for _ in range(5):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            torch.matmul(A, B, out=C)
            b.record(stream)
            b.synchronize()
            t = a.elapsed_time(b) / 1e3
            best = t if best is None else min(best, t)
        LIVE_PEAKS["tf32_gemm"] = 2.0 * n ** 3 / best / 1e12
        del A, B, C
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return dict(LIVE_PEAKS)


def roofline_peak(mode):
    """(bound, peak TFLOP/s, basis) for the convolution kernels of a form (not the FFT comparator)."""
    if mode == "fp32":
        return "alu", FP32_PEAK_TFLOPS, "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz (FFMA, nominal)"
    bf16, src = measured_peaks()
    if mode == "tf32":
        if "tf32_gemm" in LIVE_PEAKS:
            return "tensor", LIVE_PEAKS["tf32_gemm"], "cuBLAS TF32 dense GEMM burst (8192^3) measured in this run"
        return "tensor", bf16 * 1.1 / 2.25, "TF32 dense = %s BF16 peak %.1f x nominal ratio 1.1/2.25" % (src, bf16)
    return "tensor", bf16, "%s BF16 dense peak (cuBLAS burst)" % src


WORKLOADS = {
    "ring3d": "X 512x512x128 filaments (320), H 31x31x21 Gaussian-plus-ring, Y = X (*) H + Poisson noise",
    "fil3d": "X 256x256x64 filaments (40) + background 10, H 15x15x11 Gaussian sigma (1.5,1.5,3), Poisson noise",
    "blobs2d": "X 64x64 Gaussian blobs (20), H 7x7 Gaussian sigma 1.5, Gaussian noise 0.01",
    "grad3d": "4 filament volumes 128x128x64, H 11x11x9 Gaussian sigma (1.5,1.5,3): forward, dX and dH",
    "batch64": "64 filament volumes, sizes U[32,256]^2 x U[16,128], odd templates U[5,21] per axis, "
               "Gaussian sigma U[0.8,4], Poisson noise; solved together (batched solver)",
}
METRIC = "GMAC/s of projected-gradient deconvolution (forward + adjoint direct convolution per iteration)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cdv", choices=["cdv", "reference"])
    ap.add_argument("--workload", default="ring3d", choices=sorted(WORKLOADS))
    ap.add_argument("--mode", default="split3", choices=["fp32", "bf16", "tf32", "split3", "fft", "separable"],
                    help="arithmetic of the convolutions (default: split-BF16x3, the fastest form within the FP32 "
                         "accuracy bar; fft: the cuFFT comparator, not the paper's method; separable: the "
                         "template as 1-D factors, --kernels-only on the Gaussian workloads)")
    ap.add_argument("--no-forms", action="store_true", help="skip the per-form kernel timings and errors")
    ap.add_argument("--path", default="auto", choices=["auto", "general", "small"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch the iteration's kernels on the stream instead of replaying the CUDA graph "
                         "(the same kernels; for profilers that do not follow conditional graph nodes)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-sample-planes", type=int, default=96)
    ap.add_argument("--forms-iter", default=None, metavar="REF.npz",
                    help="run every form's K-step iteration and compare it with the FP64 oracle's result in "
                         "REF.npz (written by oracle/make_refs.py)")
    ap.add_argument("--kernels-only", action="store_true",
                    help="time the forward and adjoint kernels alone (launch order: forward, adjoint, forward, adjoint)")
    return ap.parse_args()


def problem(name):
    import synth
    return {"ring3d": synth.ring3d, "fil3d": synth.fil3d, "blobs2d": synth.blobs2d, "batch64": synth.batch64}[name]()


# Gaussian templates of the workloads, as (samples, sigma) per axis: their 1-D factors for the separable mode
SEPARABLE = {"fil3d": ((15, 15, 11), (1.5, 1.5, 3.0)), "blobs2d": ((7, 7), (1.5, 1.5))}


def set_template(pl, P, name, mode, dev):
    """The workload's template on a plan: dense, or as its 1-D factors in the separable mode."""
    import torch

    import synth
    if mode != "separable":
        pl.set_psf(torch.from_numpy(P.H).to(dev))
        return
    if name not in SEPARABLE:
        raise SystemExit("--mode separable: the %s template is not a product of 1-D factors" % name)
    q, sigma = SEPARABLE[name]
    pl.set_psf_factors([torch.from_numpy(h).to(dev) for h in synth.gaussian_factors(q, sigma)])


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------- CPU oracle
def oracle_sample(P, planes):
    """Time the FP64 oracle on a slab of the workload: forward + residual + adjoint + update."""
    import oracle
    m1 = min(planes, P.m[0]) if len(P.m) == 3 else P.m[0]
    X = np.ascontiguousarray(P.X_true[:m1]).astype(np.float64)
    Ys = oracle.forward(X[:1], P.H)          # touch the library (build/load) outside the clock
    del Ys
    Y = np.ascontiguousarray(P.Y[:m1 + P.H.shape[0] - 1]).astype(np.float64)
    t0 = time.perf_counter()
    R = oracle.forward(X, P.H) - Y
    G = oracle.adjoint(R, P.H)
    Xn = np.maximum(X - G, 0.0)
    dt = time.perf_counter() - t0
    del Xn
    mac = 2.0 * X.size * P.H.size
    return {"seconds": dt, "gmac": mac / 1e9, "planes": m1, "threads": oracle.num_threads()}


def cpu_model():
    """The host CPU's model name (lscpu), else the machine type."""
    import platform
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.machine()


def cpu_baseline(P, planes):
    """The FP64 oracle on all host cores, and on one thread over a sixteenth of the slab."""
    import oracle
    s = oracle_sample(P, planes)
    nxnh = float(np.prod(P.m)) * float(P.H.size)
    rate = s["gmac"] / s["seconds"]
    threads = oracle.num_threads()
    oracle.set_num_threads(1)
    try:
        s1 = oracle_sample(P, max(1, planes // 16))
    finally:
        oracle.set_num_threads(threads)
    return {"value": rate, "unit": "GMAC/s", "cores": s["threads"], "kind": "oracle",
            "iters_per_s": rate * 1e9 / (2.0 * nxnh), "cpu_model": cpu_model(),
            "sample": "FP64 oracle forward + residual + adjoint + update on planes [0, %d) of axis 1 "
                      "(%.3g GMAC, %.1f s)" % (s["planes"], s["gmac"], s["seconds"]),
            "single_thread": {"value": s1["gmac"] / s1["seconds"], "unit": "GMAC/s", "cores": s1["threads"],
                              "sample": "planes [0, %d) (%.3g GMAC, %.1f s)" % (s1["planes"], s1["gmac"],
                                                                              s1["seconds"])}}


# ---------------------------------------------------------------- clocks
class Clocks:
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.rows = []
        if self.p is None:
            return
        time.sleep(0.25)
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out = ""
        for line in out.strip().splitlines():
            f = [v.strip() for v in line.split(",")]
            if len(f) >= 8:
                self.rows.append(f)

    def summary(self):
        rows = getattr(self, "rows", [])
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[0]) for r in rows if num(r[0]) is not None]
        mx = [num(r[1]) for r in rows if num(r[1]) is not None]
        pw = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- GPU arm
def kernel_hash(mode):
    h = hashlib.sha256()
    for f in (("conv_fp32.cuh",) if mode == "fp32" else ("conv_tc.cuh", "conv_tc.cu", "conv_tc4.cuh", "conv_tc4.cu")):
        h.update(open(os.path.join(ROOT, "paper_1711_11224_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def traffic_record(workload, mode, kernel):
    """DRAM bytes per launch from a committed ncu capture, or None if the kernel changed since."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))
        e = rec[workload][mode][kernel]
        if e.get("source_hash") != kernel_hash(mode):
            return None
        return float(e["bytes_per_launch"])
    except Exception:
        return None


def kernel_hashes():
    """Source hashes of the two convolution engines, as forms_iter records them."""
    return {"fp32": kernel_hash("fp32"), "tc": kernel_hash("split3")}


def forms_iter_record(workload):
    """The full-size 100-step comparison of every form with the FP64 oracle (bench.py --forms-iter), if it
    was recorded for the kernels as they are now; None otherwise."""
    path = os.path.join(ROOT, "profiles", "forms_iter_%s.json" % workload)
    try:
        rec = json.load(open(path))
    except Exception:
        return None
    if rec.get("kernel_hashes") != kernel_hashes():
        return None
    rec["source"] = "recorded by bench.py --forms-iter (profiles/forms_iter_%s.json)" % workload
    return rec


def run_forms_iter(args):
    """Every form's K-step iteration on the workload against the FP64 oracle's K steps from the same start
    (the centre crop of Y), read from the file that oracle/make_refs.py wrote (its input hash is checked):
    relative L2 of x_K, the largest relative error of f_0..f_K, accepted and rejected trials."""
    import importlib.util

    import torch

    from paper_1711_11224_gb300 import Plan
    spec = importlib.util.spec_from_file_location("make_refs", os.path.join(ROOT, "oracle", "make_refs.py"))
    mr = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mr)
    import synth
    ref = np.load(args.forms_iter)
    # the stored inputs (the generator may differ in the last bits between machines), checked against
    # the hash the oracle's run recorded
    P = synth.Problem(args.workload, np.zeros(1, np.float32), ref["H"], ref["Y"], int(ref["K"]))
    if str(ref["input_sha256"]) != mr.input_sha256(P):
        raise SystemExit("--forms-iter: %s: the stored inputs do not match their hash" % args.forms_iter)
    P = synth.Problem(args.workload, np.zeros(tuple(a - q + 1 for a, q in zip(P.Y.shape, P.H.shape)), np.float32),
                      P.H, P.Y, P.K)
    K = int(P.K)
    Xr = ref["X"].astype(np.float64)
    fr = ref["f"]
    dev = torch.device("cuda", 0)
    Y = torch.from_numpy(P.Y).to(dev)
    res = {"workload": "%s: %s" % (args.workload, WORKLOADS[args.workload]), "K": K,
           "reference": {"accepted": int(ref["accepted"]), "rejected": int(ref["rejected"]),
                         "seconds": float(ref["seconds"]), "threads": int(ref["threads"]),
                         "stored": "float32-rounded FP64 iterate (6e-8 relative at most)"},
           "kernel_hashes": kernel_hashes(), "forms": {}}
    for mode in ("fp32", "split3", "tf32", "bf16", "fft"):
        with Plan(P.m, P.p, mode=mode) as pl:
            pl.set_psf(torch.from_numpy(P.H).to(dev))
            X, rep = pl.iterate(Y, K=K, x0="crop", max_rejects=64)
            Xg = X.cpu().numpy().astype(np.float64)
        n = min(rep["accepted"], K) + 1
        res["forms"][mode] = {"rel_l2_x": float(np.linalg.norm(Xg - Xr) / np.linalg.norm(Xr)),
                              "max_rel_err_f": float(np.max(np.abs(rep["f"][:n] - fr[:n]) / fr[:n])),
                              "accepted": rep["accepted"], "rejected": rep["rejected"], "status": rep["status"]}
        print(json.dumps({mode: res["forms"][mode]}), flush=True)
    print(json.dumps(res), flush=True)


def forms_report(P, dev, stream, npts=1000):
    """Per form: kernel times of both convolutions and their relative L2 error on sampled outputs
    against the FP64 oracle (same inputs: X_true for the forward, a seeded residual for the adjoint)."""
    import torch

    import oracle
    from paper_1711_11224_gb300 import Plan
    rng = np.random.default_rng(0)
    Rn = rng.standard_normal(P.Y.shape).astype(np.float32)
    si = np.stack([rng.integers(0, s, npts) for s in P.Y.shape], axis=1)
    ki = np.stack([rng.integers(0, s, npts) for s in P.m], axis=1)
    yo = oracle.forward_points(P.X_true, P.H, si)
    go = oracle.adjoint_points(Rn, P.H, ki)
    X = torch.from_numpy(P.X_true).to(dev)
    Rt = torch.from_numpy(Rn).to(dev)
    Y = torch.empty(P.Y.shape, device=dev, dtype=torch.float32)
    G = torch.empty(P.m, device=dev, dtype=torch.float32)
    flops = 2.0 * float(np.prod(P.m)) * float(P.H.size)
    res = {}
    for mode in ("fp32", "split3", "tf32", "bf16", "fft"):
        pl = Plan(P.m, P.p, mode=mode)
        pl.set_psf(torch.from_numpy(P.H).to(dev))
        tf = time_kernel(lambda: pl.forward(X, Y), stream, reps=2)
        ta = time_kernel(lambda: pl.adjoint(Rt, G), stream, reps=2)
        Yh = Y.cpu().numpy()
        Gh = G.cpu().numpy()
        ef = float(np.linalg.norm(Yh[tuple(si.T)] - yo) / np.linalg.norm(yo))
        ea = float(np.linalg.norm(Gh[tuple(ki.T)] - go) / np.linalg.norm(go))
        res[mode] = {"forward_ms": tf * 1e3, "adjoint_ms": ta * 1e3,
                     "gmacs_per_conv_pair": flops / (tf + ta) / 1e9,
                     "rel_l2_forward": ef, "rel_l2_adjoint": ea,
                     "sample": "%d sampled outputs per operator vs the FP64 oracle" % npts}
        if mode == "fft":
            res[mode]["note"] = ("comparator, not the paper's method: cuFFT transforms of the zero-padded grid; "
                                 "gmacs_per_conv_pair counts the direct sums it replaces")
        else:
            bound, peak, _ = roofline_peak(mode)
            res[mode].update({"forward_frac": flops / tf / 1e12 / peak, "adjoint_frac": flops / ta / 1e12 / peak,
                              "bound": bound})
        pl.close()
    return res


def separable_report(dev, stream, npts=1000):
    """Separable-template mode on the filament workload, whose Gaussian template is given by its three
    1-D factors, beside the direct FP32 form on the same template: the workload's K-step iteration
    (iterations/s), both operators (ms; bytes the three passes read and write, against the measured HBM
    copy bandwidth) and the relative L2 error of sampled outputs against the FP64 oracle."""
    import torch

    import oracle
    import synth
    from paper_1711_11224_gb300 import Plan
    P = synth.fil3d()
    q, sigma = SEPARABLE["fil3d"]
    hs = synth.gaussian_factors(q, sigma)
    H = np.multiply.outer(np.multiply.outer(hs[0].astype(np.float64), hs[1]), hs[2])
    rng = np.random.default_rng(0)
    Rn = rng.standard_normal(P.Y.shape).astype(np.float32)
    si = np.stack([rng.integers(0, s, npts) for s in P.Y.shape], axis=1)
    ki = np.stack([rng.integers(0, s, npts) for s in P.m], axis=1)
    yo = oracle.forward_points(P.X_true, H, si)
    go = oracle.adjoint_points(Rn, H, ki)
    X = torch.from_numpy(P.X_true).to(dev)
    Rt = torch.from_numpy(Rn).to(dev)
    Yt = torch.from_numpy(P.Y).to(dev)
    Yo = torch.empty(P.Y.shape, device=dev, dtype=torch.float32)
    G = torch.empty(P.m, device=dev, dtype=torch.float32)
    m = P.m
    b = tuple(a + 2 * c for a, c in zip(P.m, P.p))
    # floats each pass reads + writes (forward: axis 3, 2, 1; adjoint: axis 1, 2, 3)
    fwd_floats = (m[0] * m[1] * m[2] + m[0] * m[1] * b[2]) + (m[0] * m[1] * b[2] + m[0] * b[1] * b[2]) + \
                 (m[0] * b[1] * b[2] + b[0] * b[1] * b[2])
    adj_floats = (b[0] * b[1] * b[2] + m[0] * b[1] * b[2]) + (m[0] * b[1] * b[2] + m[0] * m[1] * b[2]) + \
                 (m[0] * m[1] * b[2] + m[0] * m[1] * m[2])
    hbm, src = measured_hbm()
    macs = float(np.prod(P.m)) * float(np.prod(q))
    res = {"workload": "fil3d: " + WORKLOADS["fil3d"],
           "template": "15x15x11 Gaussian sigma (1.5, 1.5, 3) as three 1-D factors (outer product = the template)",
           "K": P.K}
    for mode in ("separable", "fp32"):
        pl = Plan(P.m, P.p, mode=mode)
        if mode == "separable":
            pl.set_psf_factors([torch.from_numpy(h).to(dev) for h in hs])
        else:
            pl.set_psf(torch.from_numpy(H.astype(np.float32)).to(dev))
        Xi, rep = pl.iterate(Yt, K=P.K, x0="crop")                 # graph captured outside the clock
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        Xi, rep = pl.iterate(Yt, Xi, K=P.K, x0="crop", report=False)
        e.record(stream)
        e.synchronize()
        t_it = a.elapsed_time(e) / 1e3
        tf = time_kernel(lambda: pl.forward(X, Yo), stream, reps=5)
        ta = time_kernel(lambda: pl.adjoint(Rt, G), stream, reps=5)
        r = {"ms_per_iteration": t_it / P.K * 1e3, "iters_per_s": P.K / t_it,
             "dense_equivalent_gmacs": 2 * macs * P.K / t_it / 1e9,
             "forward_ms": tf * 1e3, "adjoint_ms": ta * 1e3}
        if mode == "separable":
            Yh = Yo.cpu().numpy()
            Gh = G.cpu().numpy()
            r.update({"rel_l2_forward": float(np.linalg.norm(Yh[tuple(si.T)] - yo) / np.linalg.norm(yo)),
                      "rel_l2_adjoint": float(np.linalg.norm(Gh[tuple(ki.T)] - go) / np.linalg.norm(go)),
                      "sample": "%d sampled outputs per operator vs the FP64 oracle (dense outer-product H)" % npts,
                      "pass_bytes_forward": 4 * fwd_floats, "pass_bytes_adjoint": 4 * adj_floats,
                      "forward_gbs": 4 * fwd_floats / tf / 1e9, "adjoint_gbs": 4 * adj_floats / ta / 1e9,
                      "forward_frac_hbm": 4 * fwd_floats / tf / 1e9 / hbm,
                      "adjoint_frac_hbm": 4 * adj_floats / ta / 1e9 / hbm,
                      "peak_basis": "%s HBM copy bandwidth %.0f GB/s (intermediates of 20 MB can be served by L2)"
                                    % (src, hbm),
                      "executed_macs": pl.describe()["executed_macs"]})
        res[mode] = r
        pl.close()
    res["speedup_vs_direct_fp32"] = res["fp32"]["ms_per_iteration"] / res["separable"]["ms_per_iteration"]
    return res


def snr_db(x, ref):
    """SNR of a restoration x against the true object: 10 log10(||ref||^2 / ||x - ref||^2)."""
    ref = np.asarray(ref, dtype=np.float64)
    err = np.asarray(x, dtype=np.float64) - ref
    return float(10.0 * np.log10(np.sum(ref ** 2) / np.sum(err ** 2)))


def snr_comparison(dev):
    """The paper's qualitative comparison (Results, Figs. 1-2) on synthetic data: the projected-gradient
    NNLS iteration and Richardson-Lucy, same observation, same iteration count, same start (the centre
    crop of Y, clipped at 1e-6 for Richardson-Lucy, which needs x > 0), both on the GPU (FP32 engine).
    Richardson-Lucy divides by A x and assumes y >= 0: it gets max(Y, 0) (additive Gaussian noise on a
    zero background makes some samples of Y negative)."""
    import torch

    import synth
    from paper_1711_11224_gb300 import Plan
    res = {"definition": "SNR = 10 log10(||x_true||^2 / ||x - x_true||^2) in dB; Richardson-Lucy on max(Y, 0)"}
    for name in ("blobs2d", "fil3d"):
        P = getattr(synth, name)()
        Y = torch.from_numpy(P.Y).to(dev)
        crop = tuple(slice(p, p + m) for p, m in zip(P.p, P.m))
        x0 = np.maximum(P.Y[crop], 0.0).astype(np.float32)
        with Plan(P.m, P.p) as pl:
            pl.set_psf(torch.from_numpy(P.H).to(dev))
            X = torch.from_numpy(x0.copy()).to(dev)
            X, rep = pl.iterate(Y, X, K=P.K)
            xn = X.cpu().numpy()
            Xr = torch.from_numpy(np.maximum(x0, 1e-6)).to(dev)
            pl.richardson_lucy(torch.clamp(Y, min=0.0), Xr, P.K)
            pl.sync()
            xr = Xr.cpu().numpy()
        res[name] = {"iterations": P.K, "observation_crop": snr_db(x0, P.X_true), "nnls_projected_gradient": snr_db(xn, P.X_true),
                     "richardson_lucy": snr_db(xr, P.X_true), "nnls_status": rep["status"]}
    return res


def time_kernel(fn, stream, reps=3):
    import torch
    fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / reps / 1e3


def run_kernels_only(args):
    import torch
    from paper_1711_11224_gb300 import Plan
    P = problem(args.workload)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    pl = Plan(P.m, P.p, mode=args.mode)
    set_template(pl, P, args.workload, args.mode, dev)
    X = torch.from_numpy(P.X_true).to(dev)
    R = torch.empty(P.Y.shape, device=dev, dtype=torch.float32)
    G = torch.empty(P.m, device=dev, dtype=torch.float32)
    pl.forward(X, R)                              # warm-up launches: forward, adjoint
    pl.adjoint(R, G)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record(stream)
    pl.forward(X, R)                              # timed launches: forward, adjoint
    ev[1].record(stream)
    pl.adjoint(R, G)
    ev[2].record(stream)
    ev[2].synchronize()
    tf = ev[0].elapsed_time(ev[1]) / 1e3
    ta = ev[1].elapsed_time(ev[2]) / 1e3
    flops = 2.0 * float(np.prod(P.m)) * float(P.H.size)
    print(json.dumps({"workload": args.workload, "forward_ms": tf * 1e3, "adjoint_ms": ta * 1e3,
                      "forward_tflops": flops / tf / 1e12, "adjoint_tflops": flops / ta / 1e12}), flush=True)
    pl.close()


def run_grad(args):
    """Differentiation workload: Y = X (*) H for a batch of 4 volumes, then the backward pass
    dX = A^T dY (the adjoint kernel) and dH = sum_b sum_k X_b(k) dY_b(k + j) (the template-gradient
    kernel), as ConvFn runs them.  A step is forward + dX + dH for the whole batch; GMAC counts all three
    (each B x prod(m) x prod(2p+1) multiply-adds).  The FP64 oracle does the same on the host cores."""
    import torch

    import oracle
    import synth
    from paper_1711_11224_gb300 import Plan
    from paper_1711_11224_gb300.autograd import conv
    Xs, H, sigma = synth.grad3d()
    B = Xs.shape[0]
    m = Xs.shape[1:]
    p = tuple((q - 1) // 2 for q in H.shape)
    ny = tuple(a + 2 * b for a, b in zip(m, p))
    rng = np.random.default_rng(0)
    dYh = rng.standard_normal((B,) + ny).astype(np.float32)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    X = torch.from_numpy(Xs).to(dev)
    dY = torch.from_numpy(dYh).to(dev)
    Hd = torch.from_numpy(H).to(dev)
    pl = Plan(m, p)
    pl.set_psf(Hd)
    Y = torch.empty((B,) + ny, device=dev)
    dX = torch.empty_like(X)
    dH = torch.empty(H.shape, device=dev)

    def step():
        pl.forward(X, Y)
        pl.adjoint(dY, dX)
        pl.grad_psf(X, dY, dH)
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    K = args.steps
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(0) as clk:
        ev0.record(stream)
        for _ in range(K):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    t = ev0.elapsed_time(ev1) / 1e3
    macs = float(B) * float(np.prod(m)) * float(H.size)
    tf = time_kernel(lambda: pl.forward(X, Y), stream, reps=5)
    ta = time_kernel(lambda: pl.adjoint(dY, dX), stream, reps=5)
    tg = time_kernel(lambda: pl.grad_psf(X, dY, dH), stream, reps=5)
    pl.sync()
    # accuracy of the three results against the FP64 oracle (same inputs)
    t0 = time.perf_counter()
    yo = np.stack([oracle.forward(Xs[b], H) for b in range(B)])
    dxo = np.stack([oracle.adjoint(dYh[b], H) for b in range(B)])
    dho = oracle.grad_psf(Xs, dYh, H.shape)
    tor = time.perf_counter() - t0
    rel = lambda a, b: float(np.linalg.norm(a.astype(np.float64) - b) / np.linalg.norm(b))
    err = {"forward": rel(Y.cpu().numpy(), yo), "dX": rel(dX.cpu().numpy(), dxo), "dH": rel(dH.cpu().numpy(), dho)}
    peaks = measure_peaks(stream)
    fl = 2.0 * macs
    out = {"metric": "GMAC/s of the differentiable convolution (forward + dX + dH per batch)", "value": 3 * macs * K / t / 1e9,
           "unit": "GMAC/s", "n_gpus": 1, "steps": K, "warmup": max(3, args.warmup), "ms_per_step": t * 1e3 / K,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "grad3d: 4 filament volumes 128x128x64 (10 filaments each), H 11x11x9 Gaussian "
                                  "sigma (1.5, 1.5, 3), dY standard normal (seeded)",
                      "step": "forward (batch 4) + adjoint dX (batch 4) + template gradient dH",
                      "l2": "inputs %.0f MB + %.0f MB (X, dY), below L2 between steps" % (Xs.nbytes / 1e6, dYh.nbytes / 1e6)},
           "kernels_ms": {"forward": tf * 1e3, "dX": ta * 1e3, "dH": tg * 1e3},
           "roofline": {"bound": "alu", "kernel": "grad_psf_kernel (dH)", "achieved": fl / tg / 1e12,
                        "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": fl / tg / 1e12 / FP32_PEAK_TFLOPS,
                        "frac_of_measured_ffma": fl / tg / 1e12 / peaks["fp32_ffma"], "traffic": None,
                        "forward_frac": fl / tf / 1e12 / FP32_PEAK_TFLOPS, "dX_frac": fl / ta / 1e12 / FP32_PEAK_TFLOPS,
                        "achieved_is": "2 x B x prod(m) x prod(2p+1) flop / kernel time (CUDA events)"},
           "rel_l2_vs_oracle": err, "gpu_launches": K * 4, "clocks": clk.summary(),
           "cpu_baseline": {"value": 3 * macs / tor / 1e9, "unit": "GMAC/s", "cores": oracle.num_threads(),
                            "kind": "oracle", "sample": "the whole batch: FP64 oracle forward, adjoint and grad_psf "
                                                        "(%.1f s)" % tor},
           "measured_peaks": peaks}
    # end to end through the public autograd API: X from pinned host memory, loss and dH back
    Xh = torch.empty(X.shape, dtype=torch.float32, pin_memory=True)
    Xh.copy_(torch.from_numpy(Xs))
    W = dY

    def e2e_step():
        Xd = Xh.to(dev, non_blocking=True).requires_grad_(True)
        Hg = Hd.clone().requires_grad_(True)
        loss = (conv(Xd, Hg) * W).sum()
        loss.backward()
        return float(loss.item()), Hg.grad.cpu()
    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(K):
        e2e_step()
    te = time.perf_counter() - t0
    out["e2e"] = {"value": 3 * macs * K / te / 1e9, "unit": "GMAC/s", "h2d_bytes_per_step": int(Xs.nbytes),
                  "d2h_bytes_per_step": 8 + int(H.nbytes), "seconds": te,
                  "call": "paper_1711_11224_gb300.conv (ConvFn) forward + loss.backward(): X copied in, the loss "
                          "and dH copied out every step"}
    pl.close()
    print(json.dumps(out), flush=True)


def run_batch(args):
    """Batched solver on the 64-volume workload, against the same volumes solved one after another."""
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl", device_id=torch.device("cuda", local))
    from paper_1711_11224_gb300 import BatchPlan, Plan
    from paper_1711_11224_gb300.shard import lpt_assign, volume_cost
    probs = problem("batch64")
    if ws > 1:                                        # each rank solves its LPT share of the 64 volumes
        mine = lpt_assign([volume_cost(P.m, P.H.shape) for P in probs], ws)[rank]
        probs = [probs[i] for i in mine]
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    K = args.steps
    Ys = [torch.from_numpy(P.Y).to(dev) for P in probs]
    Xs = [torch.empty(P.m, device=dev, dtype=torch.float32) for P in probs]
    bp = BatchPlan([P.m for P in probs], [P.p for P in probs], autotune=True)
    bp.set_psfs([torch.from_numpy(P.H).to(dev) for P in probs])
    done = 0
    while done < max(1, args.warmup):
        bp.iterate(Ys, Xs, K=K, x0="crop")
        done += K
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record(stream)
        _, reps = bp.iterate(Ys, Xs, K=K, x0="crop", use_graph=not args.no_graph)
        ev1.record(stream)
        torch.cuda.synchronize()
    t = ev0.elapsed_time(ev1) / 1e3
    if dist:
        tt = torch.tensor([t], device=dev, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    gmac = sum(r["gmac"] for r in reps)
    acc = min(r["accepted"] for r in reps)
    if dist:
        g = torch.tensor([gmac], device=dev, dtype=torch.float64)
        dist.all_reduce(g, op=dist.ReduceOp.SUM)
        gmac = float(g.item())
    # the same run through common trial slots of batched launches (path="general"), for comparison
    bp.iterate(Ys, Xs, K=K, x0="crop", path="general")
    torch.cuda.synchronize()
    ev0.record(stream)
    _, reps_slot = bp.iterate(Ys, Xs, K=K, x0="crop", path="general", use_graph=not args.no_graph)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_slot = ev0.elapsed_time(ev1) / 1e3
    # the plain form: each volume alone through cdv_iterate (general path, its own graph), back to back
    seq = 0.0
    for P, Y, X in zip(probs, Ys, Xs):
        with Plan(P.m, P.p) as pl:
            pl.set_psf(torch.from_numpy(P.H).to(dev))
            pl.iterate(Y, X, K=K, x0="crop", path="general")
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pl.iterate(Y, X, K=K, x0="crop", path="general", report=False)
            e1.record(stream)
            e1.synchronize()
            seq += e0.elapsed_time(e1) / 1e3
    nconv = len(probs) * (1 + 2 * K)
    ng = len({P.H.shape[-1] for P in probs})          # one batched launch per template width per convolution
    trials = max(r["trials"] for r in reps_slot)
    # persistent run: x0, state, the persistent kernel, finalize (and three memsets).  Slot path: x0, state,
    # forward per width, decision, then per trial slot: adjoint and forward per width, decision, loop
    # condition; finalize
    launches = 4
    launches_slot = 1 + 1 + ng + 1 + trials * (2 * ng + 2) + 1
    out = {"metric": METRIC, "value": gmac / t, "unit": "GMAC/s", "n_gpus": ws, "steps": K,
           "warmup": args.warmup, "ms_per_step": t * 1e3 / max(1, acc), "higher_is_better": True,
           "scaling": "strong" if ws > 1 else "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "batch64: " + WORKLOADS["batch64"], "mode": "fp32", "volumes": len(probs),
                      "K_per_call": K, "accepted_min": acc, "all_ok": all(r["status"] == "CDV_OK" for r in reps),
                      "l2": "inputs larger than L2 (%.0f MB of Y)" % (sum(P.Y.nbytes for P in probs) / 1e6)},
           "iters_per_s": acc / t, "gpu_launches": launches,
           "run": "one persistent launch for every volume's whole run (cdv_batch_iterate, path persistent)",
           "slot_path": {"value": sum(r["gmac"] for r in reps_slot) / t_slot, "unit": "GMAC/s", "seconds": t_slot,
                         "gpu_launches": launches_slot, "speedup_vs_sequential": None,
                         "call": "cdv_batch_iterate, path general: common trial slots of batched launches"},
           "sequential_plain": {"value": sum(r["gmac"] for r in reps) / seq, "unit": "GMAC/s", "seconds": seq,
                                "call": "cdv_iterate per volume (general path), back to back"},
           "batched_speedup": seq / t, "convolutions": nconv, "clocks": clk.summary()}
    out["slot_path"]["speedup_vs_sequential"] = seq / t_slot
    bp.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def run_cdv(args):
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl", device_id=torch.device("cuda", local))
    from paper_1711_11224_gb300 import Plan
    P = problem(args.workload)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    Y = torch.from_numpy(P.Y).to(dev)
    H = torch.from_numpy(P.H).to(dev)
    X = torch.empty(P.m, device=dev, dtype=torch.float32)
    pl = Plan(P.m, P.p, mode=args.mode)
    pl.set_psf(H)
    K = args.steps
    nxnh = float(np.prod(P.m)) * float(P.H.size)

    # warm-up: at least W steps, and the K-step graph captured outside the clock
    done = 0
    while True:
        _, rep = pl.iterate(Y, X, K=K, x0="crop", path=args.path, use_graph=not args.no_graph)
        done += K
        if done >= args.warmup:
            break
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record(stream)
        _, rep = pl.iterate(Y, X, K=K, x0="crop", path=args.path, use_graph=not args.no_graph)
        ev1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t = ev0.elapsed_time(ev1) / 1e3
    if dist:
        tt = torch.tensor([t], device=dev, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    gmac_rank = rep["gmac"]
    value = gmac_rank * ws / t
    iters = rep["accepted"] * ws / t
    # one graph: x0, [x0 shadow], state, initial forward, initial decision, then a WHILE loop of trial
    # slots (adjoint, forward, decision: 3 launches per trial), finalize
    # (launched on the stream instead, every one of the K + 16 trial slots is launched; spare ones
    # return at once)
    slots = rep["trials"] if not args.no_graph else K + 16
    if args.mode == "fft":
        # our kernels only (cuFFT's own are not counted): per operator pad, spectrum product, crop with
        # the fused epilogue
        launches = 1 + 1 + 3 + 1 + slots * (3 + 3 + 1) + 1
    else:
        # x0, its input shadow(s) (the narrow tensor-core kernel reads two copies), state, initial forward,
        # initial decision, 3 per trial slot, finalize
        shadows = 0 if args.mode == "fp32" else (2 if pl.describe()["cols"][0] == 4 else 1)
        launches = 1 + shadows + 1 + 1 + 1 + 3 * slots + 1

    dtype = {"fp32": "f32", "split3": "bf16x3 (split FP32, FP32 accumulate)", "tf32": "tf32 (FP32 accumulate)",
             "fft": "f32 (cuFFT comparator)",
             "bf16": "bf16 (FP32 accumulate)"}[args.mode]
    out = {"metric": METRIC, "value": value, "unit": "GMAC/s", "n_gpus": ws, "steps": K, "warmup": args.warmup,
           "ms_per_step": t * 1e3 / max(1, rep["accepted"]), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": dtype, "data": "synthetic",
           "config": {"workload": "%s: %s" % (args.workload, WORKLOADS[args.workload]), "mode": args.mode,
                      "path": args.path,
                      "K_per_call": K, "accepted": rep["accepted"], "rejected": rep["rejected"],
                      "status": rep["status"], "parallelism": "independent problem per GPU" if ws > 1 else "1 GPU",
                      "l2": "inputs larger than L2 (Y %.0f MB, X %.0f MB > 129 MB)"
                            % (P.Y.nbytes / 1e6, P.X_true.nbytes / 1e6)},
           "iters_per_s": iters, "gpu_launches": launches}

    # per-kernel timing of the two convolutions (CUDA events on the launching stream)
    R = torch.empty(P.Y.shape, device=dev, dtype=torch.float32)
    G = torch.empty(P.m, device=dev, dtype=torch.float32)
    Xs = X.clone()
    tf = time_kernel(lambda: pl.forward(Xs, R), stream)
    ta = time_kernel(lambda: pl.adjoint(R, G), stream)
    flops = 2.0 * nxnh
    dom, tdom = ("forward", tf) if tf >= ta else ("adjoint", ta)
    achieved = flops / tdom / 1e12
    if args.mode == "fft":
        # the comparator streams its input and output through transforms: HBM-bound; algorithmic bytes =
        # input once + output once of the operator
        hbm, _ = measured_hbm()
        byts = 4.0 * (float(np.prod(P.m)) + float(np.prod(P.Y.shape)))
        out["roofline"] = {"bound": "hbm", "achieved": byts / tdom / 1e9, "peak": hbm, "unit": "GB/s",
                           "frac": byts / tdom / 1e9 / hbm, "traffic": None, "kernel": "cuFFT convolution " + dom,
                           "forward_ms": tf * 1e3, "adjoint_ms": ta * 1e3,
                           "achieved_is": "input + output bytes of the operator / its time (pad, R2C, product, "
                                          "C2R, crop)"}
    else:
        bound, peak, basis = roofline_peak(args.mode)
        kname = ("conv_fp32 " if args.mode == "fp32" else "conv_tc<%s> " % args.mode) + dom
        traffic = traffic_record(args.workload, args.mode, dom)
        out["roofline"] = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                           "frac": achieved / peak, "traffic": traffic, "kernel": kname,
                           "forward_ms": tf * 1e3, "adjoint_ms": ta * 1e3,
                           "forward_frac": flops / tf / 1e12 / peak, "adjoint_frac": flops / ta / 1e12 / peak,
                           "peak_basis": basis,
                           "achieved_is": "algorithmic flop (2 x prod(m) x prod(2p+1)) / kernel time"}
    if args.mode not in ("fp32", "fft"):
        # tensor-pipe work of the dominant kernel as the library counts it (Toeplitz window, ragged
        # tiles, padded planes, the three products of split-BF16x3)
        info = pl.describe()
        d = 0 if dom == "forward" else 1
        ratio = info["executed_macs"][d] / info["algorithmic_macs"]
        out["roofline"]["executed_tflops"] = achieved * ratio
        out["roofline"]["executed_frac"] = achieved * ratio / peak
        out["roofline"]["executed_per_algorithmic"] = ratio
        out["roofline"]["tile"] = {"cols_per_plane": info["cols"][d], "K": info["K"][d], "grid": info["grid"][d],
                                   "tiles": info["tiles"][d]}
    out["clocks"] = clk.summary()
    if rank == 0:
        peaks = measure_peaks(stream)
        out["measured_peaks"] = {"fp32_ffma_tflops": peaks["fp32_ffma"], "tf32_gemm_tflops": peaks["tf32_gemm"],
                                 "how": "cdv_probe_fp32_fma (8 FMA chains per thread, 608 x 512 threads) and "
                                        "cuBLAS TF32 8192^3 GEMM, CUDA events, best of several, after the "
                                        "timed region"}
        if args.mode == "fp32":
            out["roofline"]["frac_of_measured_ffma"] = achieved / peaks["fp32_ffma"]
    if rank == 0 and not args.no_forms:
        out["forms"] = forms_report(P, dev, stream)
        rec = forms_iter_record(args.workload)
        if rec is not None:
            out["forms_iter"] = rec

    # end to end through the host-array C-ABI call (pinned buffers, copies inside the clock)
    if not args.no_e2e:
        Yh = torch.empty(P.Y.shape, dtype=torch.float32, pin_memory=True)
        Yh.copy_(torch.from_numpy(P.Y))
        Xh = torch.empty(P.m, dtype=torch.float32, pin_memory=True)
        Yn, Xn = Yh.numpy(), Xh.numpy()
        pl.iterate_host(Yn, Xn, K=K, x0="crop", report=False, path=args.path)   # graph captured outside the clock
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        _, rep2 = pl.iterate_host(Yn, Xn, K=K, x0="crop", path=args.path)
        te = time.perf_counter() - t0
        if dist:
            tt = torch.tensor([te], device=dev, dtype=torch.float64)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            te = float(tt.item())
        out["e2e"] = {"value": rep2["gmac"] * ws / te, "unit": "GMAC/s",
                      "h2d_bytes_per_step": int(P.Y.nbytes) / K, "d2h_bytes_per_step": int(P.X_true.nbytes) / K,
                      "h2d_bytes_per_call": int(P.Y.nbytes), "d2h_bytes_per_call": int(P.X_true.nbytes),
                      "steps_per_call": K, "seconds": te,
                      "call": "cdv_iterate_host (x0 = centre crop of Y; K steps per call: Y copied in and x_K "
                              "copied out once per call, so the per-step bytes are the per-call bytes / K)"}
    if rank == 0 and not args.no_cpu and ws == 1:
        out["cpu_baseline"] = cpu_baseline(P, args.cpu_sample_planes)
    if rank == 0 and not args.no_forms:
        out["snr_comparison"] = snr_comparison(dev)
        out["separable"] = separable_report(dev, stream)
    pl.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


# ---------------------------------------------------------------- reference arm (FP64 oracle)
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    P = problem(args.workload)
    planes = max(1, args.cpu_sample_planes // 2)
    for _ in range(args.warmup):
        oracle_sample(P, max(1, planes // 8))
    tot_s = tot_g = 0.0
    thr = 1
    for _ in range(args.steps):
        s = oracle_sample(P, planes)
        tot_s += s["seconds"]
        tot_g += s["gmac"]
        thr = s["threads"]
    rate = tot_g / tot_s
    nxnh = float(np.prod(P.m)) * float(P.H.size)
    out = {"impl": "reference", "metric": METRIC, "value": rate, "unit": "GMAC/s", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_s * 1e3 / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "%s: %s" % (args.workload, WORKLOADS[args.workload]), "mode": "oracle"},
           "iters_per_s": rate * 1e9 / (2.0 * nxnh),
           "cpu_baseline": {"value": rate, "unit": "GMAC/s", "cores": thr, "kind": "oracle",
                            "sample": "each step: FP64 oracle forward + residual + adjoint + update on planes "
                                      "[0, %d) of axis 1 of the workload" % planes},
           "e2e": {"value": rate, "unit": "GMAC/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.forms_iter:
        run_forms_iter(args)
    elif args.kernels_only:
        run_kernels_only(args)
    elif args.mode == "separable":
        raise SystemExit("--mode separable runs with --kernels-only; the default line reports the separable "
                         "iteration on fil3d under 'separable'")
    elif args.workload == "batch64":
        run_batch(args)
    elif args.workload == "grad3d":
        run_grad(args)
    else:
        run_cdv(args)


if __name__ == "__main__":
    main()
