"""Benchmark: nested dissection + approximate LDM^t factorization + FGMRES
solve to 1e-8 relative residual on one GPU per rank.

Workload (one "step" = the whole hot path on one synthetic problem):
indefinite Helmholtz -Lap u - k^2 c(x) u = f, SIPG DG p=2 on 64x64 quads
(36,864 dofs, 9x9 blocks), k for 10 dofs per wavelength, c(x) = 1 + 0.3 x
(mean of 8 random-phase cosines), Gaussian point source, ID tolerance 1e-4,
FGMRES(30) in FP64 to 1e-8.  Forms: FP64 plain (factor in FP64), mixed
(factor in FP32, FP64 Krylov) and mixed with learned sample widths (an MLP
trained before timing on the ranks of adaptive runs; the timed step includes
its BF16 inference); `value` is the first form's time to solution (default:
the learned mixed form).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Timing: CUDA events on the launching stream, a 256 MB write between timed
steps flushes L2 (129 MB), max over ranks.  Under torchrun every rank solves
its own instance (seed = rank): weak scaling, no collective in the data path.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "factor+FGMRES time to 1e-8 rel. residual (mixed vs FP64 plain, 1 GB300); apply GB/s"
WORKLOAD = "helmholtz_sipg_p2_64x64"
N_ELEM, P_DEG, TOL, RTOL, RESTART = 64, 2, 1e-4, 1e-8, 30


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--forms", default="fp32_learned,fp32,fp64",
                    help="fp32_learned: FP32 factor with learned sample widths (headline); fp32: FP32 "
                         "factor, adaptive widths; fp64: plain FP64 factor")
    ap.add_argument("--workload", default="helmholtz64",
                    choices=["helmholtz64", "batched256", "helmholtz256", "diffusion32", "gemm_update"],
                    help="helmholtz64: the timed workload (default); batched256: 256 independent "
                         "instances x 32 right-hand sides through the batched form; helmholtz256: "
                         "Helmholtz p=3 on 256x256 quads (1,048,576 dofs), learned widths; diffusion32: "
                         "3D diffusion p=1 on 32^3 hexes (262,144 dofs), 20 right-hand sides, learned "
                         "widths; gemm_update: the blocked sweep's update C += A B alone, m = n = 8192, "
                         "K = 256, FP32 (each its own JSON line)")
    ap.add_argument("--no-fp64", action="store_true",
                    help="large workloads: skip the plain FP64 comparison form")
    ap.add_argument("--tensor-cores", type=int, default=3, choices=[0, 1, 3],
                    help="GEMM engine of the FP32 forms: 0 SIMT, 1 tcgen05 (fixed rule), 3 (default) per shape "
                         "class the faster of SIMT and tcgen05, timed once (in the warm-up steps)")
    ap.add_argument("--sample-bf16", type=int, default=None, choices=[0, 1],
                    help="FP32 forms: sampling products on tcgen05 kind::f16 with S in three BF16 terms "
                         "(default: on for diffusion32, whose configuration asks for BF16 sampling; off elsewhere)")
    ap.add_argument("--probe", type=int, default=4,
                    help="residual probe vectors per accepted front in the learned-width form (0: off)")
    ap.add_argument("--quick", action="store_true",
                    help="timed steps only (no apply loop, no host-buffer run): for profiling")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return dict(hbm=d["hbm_gbs"], bf16=d["bf16_tflops"], bf16_s=d["bf16_tflops_sustained"],
                    sm_mhz=float(d.get("sm_max_mhz", 2070.0)), src="measured")
    except Exception:
        return dict(hbm=6800.0, bf16=1900.0, bf16_s=1700.0, sm_mhz=2070.0, src="fallback")


# FP32 SIMT peak from unit counts and clock: SMs (read from the device) x 128
# FP32 FMA/clk/SM x 2 flop x the maximum SM clock (from the peaks file, else
# GB300's 2,070 MHz).  FP64: the nominal 1.25 TFLOP/s of GB300.
FP64_TFLOPS = 1.25
TF32_PER_BF16 = 1.1 / 2.25   # nominal dense TF32 / BF16 rates of GB300


def with_simt_peak(pk, sms):
    """pk plus the derived FP32 SIMT peak for a device with `sms` SMs."""
    out = dict(pk)
    out["sms"] = int(sms)
    out["fp32"] = sms * 128 * 2 * pk["sm_mhz"] * 1e6 / 1e12
    out["fp32_src"] = f"derived: {sms} SMs x 128 FP32 FMA/clk x 2 x {pk['sm_mhz']:.0f} MHz"
    return out


def device_sms(dev):
    import torch
    return torch.cuda.get_device_properties(dev).multi_processor_count


def max_over_ranks(values, device):
    """Element-wise maximum of per-rank values over all ranks (the job ends
    when its slowest replica ends).  Works with any torch.distributed backend
    whose tensors live on `device`."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(list(values), device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def roofline_of(kernel, ms, cnt, work, total_ms, pk, workload=None):
    """Roofline entry of one kernel class: FLOP-counted classes (GEMMs and the
    Gauss-Jordan panels) against the FP32/FP64 arithmetic peak, byte-counted
    classes (apply, SpMV) against the measured HBM bandwidth.  pk: peaks() with
    the FP32 SIMT peak of the device (with_simt_peak)."""
    per_launch_s = ms / cnt * 1e-3
    if kernel == "gemm_tma_block":
        # the blocked sweep's K = 256 updates C += A B of whole fronts on the TMA-fed tensor-core
        # kernel: at K = 256 their arithmetic intensity against the C stream (read + write, 8 B per
        # output; A and B come from L2) is 2 * 256 / 8 = 64 flop/B, below the TF32 ridge, so HBM
        # bounds them: algorithmic bytes = flops / 64 (ragged last blocks have K < 256: an
        # underestimate of their bytes)
        tflops = work / cnt / per_launch_s / 1e12
        ach = work / 64.0 / cnt / per_launch_s / 1e9
        return dict(kernel=kernel, bound="hbm", achieved=ach, peak=pk["hbm"], unit="GB/s", frac=ach / pk["hbm"],
                    traffic=None, launches=cnt, avg_launch_us=ms / cnt * 1e3, share=ms / total_ms,
                    peak_source=f"{pk['src']} (MEASURED_PEAKS.json hbm_gbs)" if pk["src"] == "measured"
                    else pk["src"], tflops=tflops, tf32_peak_tflops=pk["bf16"] * TF32_PER_BF16,
                    tensor_frac=tflops / (pk["bf16"] * TF32_PER_BF16),
                    note="bytes = flops / 64: the C stream of K = 256 updates; A, B from L2")
    if kernel.startswith("gemm_tma") or kernel.startswith("gemm_tc"):
        peak = pk["bf16"] * TF32_PER_BF16
        ach = work / cnt / per_launch_s / 1e12
        return dict(kernel=kernel, bound="tensor", achieved=ach, peak=peak, unit="TFLOP/s", frac=ach / peak,
                    traffic=None, launches=cnt, avg_launch_us=ms / cnt * 1e3, share=ms / total_ms,
                    peak_source=f"TF32 = measured BF16 x {TF32_PER_BF16:.3f} (nominal 1.1 / 2.25 PFLOP/s)")
    if kernel.startswith("gemm") or kernel.startswith("gj_panel"):
        f32 = kernel.endswith("f32")
        peak = pk["fp32"] if f32 else FP64_TFLOPS
        ach = work / cnt / per_launch_s / 1e12
        return dict(kernel=kernel, bound="alu", achieved=ach, peak=peak, unit="TFLOP/s", frac=ach / peak,
                    traffic=profiled_traffic(kernel), launches=cnt, avg_launch_us=ms / cnt * 1e3,
                    share=ms / total_ms,
                    peak_source=pk["fp32_src"] if f32 else "nominal GB300 FP64 1.25 TFLOP/s")
    ach = work / cnt / per_launch_s / 1e9
    return dict(kernel=kernel, bound="hbm", achieved=ach, peak=pk["hbm"], unit="GB/s", frac=ach / pk["hbm"],
                traffic=profiled_traffic(kernel, workload), launches=cnt, avg_launch_us=ms / cnt * 1e3,
                share=ms / total_ms,
                peak_source=f"{pk['src']} (MEASURED_PEAKS.json hbm_gbs)" if pk["src"] == "measured"
                else pk["src"])


def profiled_traffic(kernel, workload=None):
    """DRAM bytes per launch of `kernel` from its committed ncu summary, or None
    when there is none or the kernel's source changed since the capture.  The
    apply class (one launch = one whole apply) is keyed by workload too."""
    import hashlib
    files = {"gemm_f32": ("profiles/k_gemm_f32_dram_helmholtz64_p2.md", "paper_1508_07798_gb300/csrc/gemm.cu"),
             "gj_panel_f32": ("profiles/k_gj_panel_reg_dram_helmholtz64_p2_fp32.md",
                              "paper_1508_07798_gb300/csrc/front.cu"),
             "gemm_tma": ("profiles/k_gemm_tma_gemm_update_8192x8192_k256.md",
                          "paper_1508_07798_gb300/csrc/tcgemm_tma.cu"),
             ("apply", "helmholtz64"): ("profiles/k_apply_dram_helmholtz64_p2_fp32.md",
                                        "paper_1508_07798_gb300/csrc/apply.cu")}
    key = (kernel, workload) if (kernel, workload) in files else kernel
    if key not in files:
        return None
    summary, src = (os.path.join(ROOT, f) for f in files[key])
    try:
        kv = {}
        for line in open(summary):
            if ":" in line and line.split(":")[0] in ("traffic_bytes_per_launch", "kernel_source_sha256_prefix"):
                k, v = line.split(":", 1)
                kv[k] = v.strip()
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
        if not sha.startswith(kv["kernel_source_sha256_prefix"]):
            return None
        return int(kv["traffic_bytes_per_launch"])
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.p = None
        self.lines = []

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.p = None

    def _read(self):
        for line in self.p.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1].split()[0]))
                smax = float(f[2].split()[0])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_problem(seed):
    from paper_1508_07798_gb300 import dg_inputs as dg
    mesh, A = dg.helmholtz_2d(N_ELEM, P_DEG, seed)
    b = dg.point_source_rhs(mesh, seed)[:, 0]
    return mesh, A, b


def bench_ours(args, rank, world):
    import numpy as np
    import torch
    from paper_1508_07798_gb300 import hssnd
    from paper_1508_07798_gb300 import dg_inputs as dg

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    mesh, A, b_host = make_problem(rank)
    meshdesc = (2, (N_ELEM, N_ELEM), P_DEG)
    dA = hssnd.DeviceBSR.from_host(A)
    b = torch.as_tensor(b_host, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    Acsr = dg.bsr_to_csr(A)

    # learned sample widths: the model is trained once, before any timing, on
    # the ranks of adaptive runs of the method (Helmholtz 64 x 64, p in
    # {1, 2, 3}, seeds 100..115, the same ID tolerance); the timed step then
    # includes the box features, the BF16 inference and the width read-back
    model = None
    learned_info = None
    c_elem = dg.cosine_field(mesh, rank)
    kappa_h = dg.helmholtz_kappa(N_ELEM, P_DEG) / N_ELEM
    if "fp32_learned" in args.forms.split(","):
        from paper_1508_07798_gb300 import ranks
        probs = dg.rank_training_problems(N_ELEM)
        Xt, tt = ranks.training_set(probs, tol=TOL)
        model = hssnd.RankModel(seed=1)
        model.fit_norm(Xt, tt)
        train_loss = model.train(Xt, tt, epochs=60, batch=256, lr=2e-3, seed=3)
        learned_info = dict(train_samples=int(len(tt)), train_loss=train_loss)

    def step(prec, marks=None):
        # marks: two CUDA events recorded after the ordering and after the factor
        tree = hssnd.nd_order(meshdesc, dA, leaf_max=64)
        if marks is not None:
            marks[0].record(stream)
        if prec == "fp32_learned":
            r0 = model.predict(hssnd.rank_features(tree, c_elem, kappa_h))[1]
            F = hssnd.hss_factor(dA, tree, tol=TOL, precision="fp32", r_init=r0, autotune=1, probe=args.probe,
                                 tensor_cores=args.tensor_cores, sample_bf16=args.sample_bf16 or 0)
        else:
            F = hssnd.hss_factor(dA, tree, tol=TOL, precision=prec, autotune=1,
                                 tensor_cores=args.tensor_cores if prec == "fp32" else 0,
                                 sample_bf16=(args.sample_bf16 or 0) if prec == "fp32" else 0)
        if marks is not None:
            marks[1].record(stream)
        x, st = hssnd.fgmres_solve(dA, F, b, rtol=RTOL, restart=RESTART)
        return tree, F, x, st

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    forms = {}
    launches_total = 0
    clk = Clocks(dev.index)
    prof_all = {}
    for prec in args.forms.split(","):
        for _ in range(args.warmup):
            step(prec)
        torch.cuda.synchronize()
        barrier()
        if prec == args.forms.split(",")[0]:
            clk.start()

        def timed(steps, phases=None):
            ts, lastv = [], None
            for _ in range(steps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                marks = [torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
                torch.cuda.synchronize()
                e0.record(stream)
                lastv = step(prec, marks)
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
                if phases is not None:
                    phases["nd_order"].append(e0.elapsed_time(marks[0]))
                    phases["factor"].append(marks[0].elapsed_time(marks[1]))
                    phases["fgmres"].append(marks[1].elapsed_time(e1))
            return ts, lastv

        # pass 1: the headline time, no instrumentation
        l0 = hssnd.launch_count()
        phases = {"nd_order": [], "factor": [], "fgmres": []}
        times, last = timed(args.steps, phases)
        launches_total += hssnd.launch_count() - l0
        # the factorization's host side, from the last uninstrumented step
        hinfo = last[1].info()
        host = dict(syncs=hinfo["host_syncs"], sync_wait_ms=hinfo["host_sync_ms"], call_ms=hinfo["host_ms"],
                    work_ms=hinfo["host_ms"] - hinfo["host_sync_ms"], idle_after_readback_ms=hinfo["host_gap_ms"])
        # pass 2: the same steps with every kernel launch bracketed by CUDA events
        hssnd.profile_reset()
        hssnd.profile_enable(True)
        ptimes, _ = timed(args.steps)
        hssnd.profile_enable(False)
        prof = hssnd.profile_read()
        prof_all[prec] = prof
        tree, F, x, st = last
        xr = x.cpu().numpy()
        relres = float(np.linalg.norm(b_host - Acsr @ xr) / np.linalg.norm(b_host))
        info = F.info()
        forms[prec] = dict(ms=statistics.mean(times), ms_min=min(times), ms_median=statistics.median(times),
                           ms_all=times, phases_ms={k: statistics.mean(v) for k, v in phases.items()},
                           ms_instrumented=statistics.mean(ptimes), iters=st.iters,
                           relres=relres, converged=bool(st.converged and relres <= RTOL * 1.0001),
                           factor_bytes=info["factor_bytes"], front_flops=info["front_flops"],
                           executed_flops=info["executed_flops"], max_rank=info["max_rank"], max_r=info["max_r"],
                           sampling_rounds=int(F.export_log()["rounds"].sum()),
                           probe_regrown=info["probe_regrown"], factor_host=host,
                           kernel_ms_sum=sum(v[0] for v in prof.values()) / args.steps)
    clocks = clk.stop()
    barrier()
    if args.quick:
        return dict(metric=METRIC, quick=True, forms={k: {kk: vv for kk, vv in v.items() if kk != "ms_all"}
                                                      for k, v in forms.items()},
                    gpu_launches=int(launches_total // max(1, len(forms))))

    # ---- apply GB/s: 20 applies of the last factor of each form, L2 flushed between
    apply = {}
    pk = with_simt_peak(peaks(), device_sms(dev))
    for prec in args.forms.split(","):
        if prec == "fp32_learned":
            continue      # same factor storage and apply kernels as fp32
        tree = hssnd.nd_order(meshdesc, dA, leaf_max=64)
        F = hssnd.hss_factor(dA, tree, tol=TOL, precision=prec, autotune=1)
        N = A.n
        xv = torch.randn(N, dtype=torch.float64, device=dev)
        yv = torch.empty_like(xv)
        for _ in range(3):
            hssnd.hss_apply_raw(F, 1, xv, yv, N)
        hssnd.profile_reset()
        hssnd.profile_enable(True)
        ts = []
        for _ in range(20):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            hssnd.hss_apply_raw(F, 1, xv, yv, N)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        hssnd.profile_enable(False)
        pr = hssnd.profile_read()
        byt = sum(v[2] for k, v in pr.items() if k.startswith("apply"))
        kms = sum(v[0] for k, v in pr.items() if k.startswith("apply"))
        per_apply_bytes = byt / 20
        apply[prec] = dict(ms=statistics.median(ts), bytes=per_apply_bytes,
                           gbs=per_apply_bytes / (statistics.median(ts) * 1e-3) / 1e9,
                           kernel_gbs=byt / (kms * 1e-3) / 1e9 if kms > 0 else None)
        apply[prec]["frac"] = apply[prec]["gbs"] / pk["hbm"]
        fw, bw = F.apply_plan()
        apply[prec]["work_split"] = dict(fwd=fw.tolist(), bwd=bw.tolist())

    # ---- e2e through the C ABI with host buffers: H2D of A and b, solve, D2H of x
    e2e = None
    head = args.forms.split(",")[0]
    rp = torch.as_tensor(A.row_ptr).pin_memory()
    ci = torch.as_tensor(A.col_idx).pin_memory()
    va = torch.as_tensor(A.val.reshape(-1)).pin_memory()
    bh = torch.as_tensor(b_host).pin_memory()
    xh = torch.empty_like(bh).pin_memory()
    d_rp = torch.empty_like(rp, device=dev)
    d_ci = torch.empty_like(ci, device=dev)
    d_va = torch.empty_like(va, device=dev)
    d_b = torch.empty_like(bh, device=dev)
    h2d = rp.numel() * 4 + ci.numel() * 4 + va.numel() * 8 + bh.numel() * 8
    d2h = xh.numel() * 8
    ets = []
    for it in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        d_rp.copy_(rp, non_blocking=True)
        d_ci.copy_(ci, non_blocking=True)
        d_va.copy_(va, non_blocking=True)
        d_b.copy_(bh, non_blocking=True)
        dA2 = hssnd.DeviceBSR.__new__(hssnd.DeviceBSR)
        dA2.nb, dA2.bs, dA2.row_ptr, dA2.col_idx, dA2.val = A.nb, A.bs, d_rp, d_ci, d_va
        dA2.c = hssnd.hss_bsr(A.nb, A.bs, d_rp.data_ptr(), d_ci.data_ptr(), d_va.data_ptr())
        tree = hssnd.nd_order(meshdesc, dA2, leaf_max=64)
        if head == "fp32_learned":
            r0 = model.predict(hssnd.rank_features(tree, c_elem, kappa_h))[1]
            F = hssnd.hss_factor(dA2, tree, tol=TOL, precision="fp32", r_init=r0, autotune=1, probe=args.probe,
                                 tensor_cores=args.tensor_cores, sample_bf16=args.sample_bf16 or 0)
        else:
            F = hssnd.hss_factor(dA2, tree, tol=TOL, precision=head, autotune=1,
                                 tensor_cores=args.tensor_cores if head == "fp32" else 0,
                                 sample_bf16=(args.sample_bf16 or 0) if head == "fp32" else 0)
        x, st = hssnd.fgmres_solve(dA2, F, d_b, rtol=RTOL, restart=RESTART)
        xh.copy_(x, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if it >= args.warmup:
            ets.append(e0.elapsed_time(e1))
    e2e = dict(value=statistics.mean(ets), unit="ms", h2d_bytes_per_step=int(h2d), d2h_bytes_per_step=int(d2h))

    # ---- max over ranks
    value = forms[head]["ms"]
    if world > 1:
        value, e2e["value"] = max_over_ranks([value, e2e["value"]], dev)

    # ---- roofline of the dominant kernel of the headline form
    prof = prof_all[head]
    tracked = {k: v for k, v in prof.items() if v[2] > 0}
    dom = max(tracked, key=lambda k: tracked[k][0]) if tracked else max(prof, key=lambda k: prof[k][0])
    total_ms = sum(v[0] for v in prof.values())
    roof = roofline_of(dom, *prof[dom], total_ms, pk, workload="helmholtz64")
    # the next tracked classes by time, for context
    roof["others"] = [roofline_of(k, *prof[k], total_ms, pk, workload="helmholtz64") for k in
                      sorted(tracked, key=lambda k: -tracked[k][0]) if k != dom][:3]
    kernels = {form: {k: dict(ms=round(v[0] / args.steps, 4), launches=v[1] // args.steps) for k, v in
                      sorted(pf.items(), key=lambda kv: -kv[1][0])} for form, pf in prof_all.items()}
    res = dict(metric=METRIC, value=value, unit="ms", n_gpus=world, steps=args.steps, warmup=args.warmup,
               ms_per_step=value, higher_is_better=False, scaling="weak", vs_baseline=None,
               dtype="f32 factor / f64 Krylov" if head.startswith("fp32") else "f64", data="synthetic",
               config=headline_config(args, world),
               learned_widths=learned_info if model is not None else None,
               forms={k: {kk: vv for kk, vv in v.items() if kk != "ms_all"} for k, v in forms.items()},
               apply=apply, roofline=roof, e2e=e2e, clocks=clocks, gpu_launches=int(launches_total // max(1, len(forms))),
               kernels_per_step=kernels)
    return res


# ---- the large configurations: Helmholtz p = 3 on 256 x 256 quads and 3D diffusion p = 1 on 32^3 hexes
LARGE = {
    "helmholtz256": dict(dim=2, n=256, p=3, tol=1e-6, nrhs=1, rmax=96, bf16=0,
                         workload="helmholtz_sipg_p3_256x256", small=(64, 3)),
    "diffusion32": dict(dim=3, n=32, p=1, tol=1e-5, nrhs=20, rmax=96, bf16=1,
                        workload="diffusion3d_sipg_p1_32cubed_20rhs", small=(16, 1)),
}


def large_problem(spec, seed, n=None, p=None):
    """(mesh, A, b (ndof x nrhs), mesh descriptor, c per element for the features, kappa h)."""
    from paper_1508_07798_gb300 import dg_inputs as dg
    n = spec["n"] if n is None else n
    p = spec["p"] if p is None else p
    if spec["dim"] == 2:
        mesh, A = dg.helmholtz_2d(n, p, seed)
        b = dg.point_source_rhs(mesh, seed)
        return mesh, A, b, (2, (n, n), p), dg.cosine_field(mesh, seed), dg.helmholtz_kappa(n, p) / n
    mesh, A = dg.diffusion_3d(n, p, seed)
    b = dg.random_rhs(A.n, spec["nrhs"], seed, kind="normal")
    return mesh, A, b, (3, (n, n, n), p), np.log(dg.gaussian_log_field(mesh, seed)), 0.0


def bench_large(args, rank, world):
    """One step = nd_order + hss_factor + fgmres_solve (all right-hand sides
    in lock step) of a large configuration.  Forms: FP32 factor with learned
    widths and the residual probe (headline), FP32 with adaptive widths, plain
    FP64 (unless --no-fp64).  The width model is trained before timing on the
    ranks of adaptive runs of the method on smaller problems of the same
    family (64 x 64 Helmholtz p = 1, 2, 3 or 16^3 diffusion, seeds
    100..115)."""
    import torch
    from paper_1508_07798_gb300 import hssnd
    from paper_1508_07798_gb300 import dg_inputs as dg
    from paper_1508_07798_gb300 import ranks
    spec = LARGE[args.workload]
    bf16 = spec["bf16"] if args.sample_bf16 is None else args.sample_bf16
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    mesh, A, b_host, meshdesc, c_elem, kappa_h = large_problem(spec, rank)
    dA = hssnd.DeviceBSR.from_host(A)
    B = torch.as_tensor(np.asfortranarray(b_host), device=dev)
    nrhs = b_host.shape[1]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    Acsr = dg.bsr_to_csr(A)
    tol = spec["tol"]
    probs = dg.rank_training_problems(64) if spec["dim"] == 2 else dg.diffusion_training_problems(16)
    Xt, tt = ranks.training_set(probs, tol=tol, rmax=spec["rmax"])
    model = hssnd.RankModel(seed=1)
    model.fit_norm(Xt, tt)
    train_loss = model.train(Xt, tt, epochs=60, batch=256, lr=2e-3, seed=3)
    forms = ["fp32_learned", "fp32"] + ([] if args.no_fp64 else ["fp64"])

    def step(form, marks=None):
        tree = hssnd.nd_order(meshdesc, dA, leaf_max=64)
        if marks is not None:
            marks[0].record(stream)
        if form == "fp32_learned":
            r0 = model.predict(hssnd.rank_features(tree, c_elem, kappa_h), rmax=spec["rmax"])[1]
            F = hssnd.hss_factor(dA, tree, tol=tol, precision="fp32", r_init=r0, autotune=1, probe=args.probe,
                                 rmax=spec["rmax"], tensor_cores=args.tensor_cores, sample_bf16=bf16)
        else:
            F = hssnd.hss_factor(dA, tree, tol=tol, precision=form, autotune=1, rmax=spec["rmax"],
                                 tensor_cores=args.tensor_cores if form == "fp32" else 0,
                                 sample_bf16=bf16 if form == "fp32" else 0)
        if marks is not None:
            marks[1].record(stream)
        x, st = hssnd.fgmres_solve(dA, F, B, rtol=RTOL, restart=RESTART)
        return tree, F, x, st

    out, prof_all = {}, {}
    clk = Clocks(dev.index)
    launches = 0
    for form in forms:
        steps = args.steps if form != "fp64" else 1
        warm = args.warmup if form != "fp64" else 1
        for _ in range(warm):
            step(form)
        torch.cuda.synchronize()
        if form == forms[0]:
            clk.start()
        ts, ph = [], {"nd_order": [], "factor": [], "fgmres": []}
        l0 = hssnd.launch_count()
        last = None
        for _ in range(steps):
            flush.zero_()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            torch.cuda.synchronize()
            ev[0].record(stream)
            last = step(form, ev[1:3])
            ev[3].record(stream)
            torch.cuda.synchronize()
            ts.append(ev[0].elapsed_time(ev[3]))
            ph["nd_order"].append(ev[0].elapsed_time(ev[1]))
            ph["factor"].append(ev[1].elapsed_time(ev[2]))
            ph["fgmres"].append(ev[2].elapsed_time(ev[3]))
        if form == forms[0]:
            clocks = clk.stop()
            launches = (hssnd.launch_count() - l0) // steps
        hssnd.profile_reset()
        hssnd.profile_enable(True)
        step(form)
        hssnd.profile_enable(False)
        prof_all[form] = hssnd.profile_read()
        tree, F, x, st = last
        X = x.cpu().numpy().reshape(A.n, -1)
        relres = float((np.linalg.norm(b_host - Acsr @ X, axis=0) / np.linalg.norm(b_host, axis=0)).max())
        info = F.info()
        out[form] = dict(ms=statistics.mean(ts), ms_min=min(ts), steps=steps, warmup=warm,
                         phases_ms={k: statistics.mean(v) for k, v in ph.items()}, iters_max=st.max_iters,
                         iters_total=st.iters, true_relres=relres,
                         converged=bool(st.converged and relres <= RTOL * 1.0001),
                         factor_bytes=info["factor_bytes"], front_flops=info["front_flops"],
                         executed_flops=info["executed_flops"], max_rank=info["max_rank"],
                         capped_fronts=info["capped_fronts"], probe_regrown=info["probe_regrown"],
                         sampling_rounds=int(F.export_log()["rounds"].sum()),
                         gemm_engines=dict(simt=info["gemm_simt"], tma=info["gemm_tma"],
                                           staged=info["gemm_staged"], bf16_sampling=info["gemm_bf16"]))
        del F, last
    head = forms[0]
    prof = prof_all[head]
    pk = with_simt_peak(peaks(), device_sms(dev))
    tracked = {k: v for k, v in prof.items() if v[2] > 0}
    dom = max(tracked, key=lambda k: tracked[k][0])
    total_ms = sum(v[0] for v in prof.values())
    roof = roofline_of(dom, *prof[dom], total_ms, pk)
    roof["others"] = [roofline_of(k, *prof[k], total_ms, pk) for k in
                      sorted(tracked, key=lambda k: -tracked[k][0]) if k != dom][:3]
    # e2e through host buffers: A and b in, x out
    rp = torch.as_tensor(A.row_ptr).pin_memory()
    ci = torch.as_tensor(A.col_idx).pin_memory()
    va = torch.as_tensor(A.val.reshape(-1)).pin_memory()
    bh = torch.as_tensor(np.asfortranarray(b_host).T.copy()).pin_memory()
    xh = torch.empty_like(bh).pin_memory()
    d_rp, d_ci, d_va = (torch.empty_like(t, device=dev) for t in (rp, ci, va))
    d_b = torch.empty_like(bh, device=dev)
    ets = []
    for it in range(1 + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for dst, src in ((d_rp, rp), (d_ci, ci), (d_va, va), (d_b, bh)):
            dst.copy_(src, non_blocking=True)
        dA2 = hssnd.DeviceBSR.__new__(hssnd.DeviceBSR)
        dA2.nb, dA2.bs, dA2.row_ptr, dA2.col_idx, dA2.val = A.nb, A.bs, d_rp, d_ci, d_va
        dA2.c = hssnd.hss_bsr(A.nb, A.bs, d_rp.data_ptr(), d_ci.data_ptr(), d_va.data_ptr())
        tree = hssnd.nd_order(meshdesc, dA2, leaf_max=64)
        r0 = model.predict(hssnd.rank_features(tree, c_elem, kappa_h), rmax=spec["rmax"])[1]
        F = hssnd.hss_factor(dA2, tree, tol=tol, precision="fp32", r_init=r0, autotune=1, probe=args.probe,
                             rmax=spec["rmax"], tensor_cores=args.tensor_cores, sample_bf16=bf16)
        x, st = hssnd.fgmres_solve(dA2, F, d_b.t(), rtol=RTOL, restart=RESTART)
        xh.copy_(x.t() if x.dim() == 2 else x.reshape(1, -1), non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if it >= 1:
            ets.append(e0.elapsed_time(e1))
        del F
    h2d = rp.numel() * 4 + ci.numel() * 4 + va.numel() * 8 + bh.numel() * 8
    value = out[head]["ms"]
    e2e_v = statistics.mean(ets)
    if world > 1:
        value, e2e_v = max_over_ranks([value, e2e_v], dev)
    kernels = {form: {k: dict(ms=round(v[0], 3), launches=v[1]) for k, v in
                      sorted(pf.items(), key=lambda kv: -kv[1][0])[:12]} for form, pf in prof_all.items()}
    return dict(metric=METRIC, value=value, unit="ms", n_gpus=world, steps=out[head]["steps"],
                warmup=out[head]["warmup"], ms_per_step=value, higher_is_better=False, scaling="weak",
                vs_baseline=None, dtype="f32 factor / f64 Krylov", data="synthetic",
                config=dict(workload=spec["workload"], dofs=A.n, p=spec["p"], dim=spec["dim"], id_tol=tol,
                            rtol=RTOL, restart=RESTART, rhs=nrhs, leaf_max=64, rmax=spec["rmax"],
                            headline_form=head, tensor_cores=args.tensor_cores, sample_bf16=bf16,
                            learned_widths=dict(train_samples=int(len(tt)), train_loss=train_loss,
                                                trained_on="adaptive runs, " + (
                                                    "Helmholtz 64x64 p=1,2,3" if spec["dim"] == 2 else
                                                    "3D diffusion 16^3 p=1") + ", seeds 100..115"),
                            learned_probe_vectors=args.probe,
                            l2="flushed by a 256 MB write before every timed step (the factor is GBs)",
                            parallelism=f"replicas x{world} (independent instances)"),
                forms=out, roofline=roof, clocks=clocks, gpu_launches=int(launches), kernels=kernels,
                tuner=hssnd.gemm_tuner_choices() if args.tensor_cores == 3 else None,
                e2e=dict(value=e2e_v, unit="ms", h2d_bytes_per_step=int(h2d), d2h_bytes_per_step=int(bh.numel() * 8)))


def bench_gemm_update(args, rank, world):
    """The GEMM of the blocked Gauss-Jordan sweep's block updates, alone:
    C += A B in FP32 with m = n = 8192 (C is 256 MB, beyond L2), K = 256
    (eight 32-column panels), through hss_gemm_f32 on the SIMT engine and on
    the TMA-fed tcgen05 engine (TF32 hi/lo split).  Per engine: kernel time by
    CUDA events (library instrumentation), TFLOP/s and the C stream's GB/s
    (read + write, 8 bytes per output: the HBM bound of this shape)."""
    import torch
    from paper_1508_07798_gb300 import hssnd
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    m = n = 8192
    k = 256
    g = torch.Generator(device="cpu").manual_seed(rank)
    A = torch.randn(n, k, generator=g).to(dev)   # row-major n x k: the column-major k x n operand B^t
    B = torch.randn(k, m, generator=g).to(dev)
    C = torch.randn(n, m, generator=g).to(dev)
    pk = with_simt_peak(peaks(), device_sms(dev))
    out = {}
    for name, eng in (("simt", 0), ("tma_tf32_split", 3)):
        for _ in range(args.warmup):
            hssnd.gemm_f32(A, B, C, alpha=1.0, beta=1.0, engine=eng)
        hssnd.profile_reset()
        hssnd.profile_enable(True)
        for _ in range(args.steps):
            hssnd.gemm_f32(A, B, C, alpha=1.0, beta=1.0, engine=eng)
        hssnd.profile_enable(False)
        pr = hssnd.profile_read()
        ms = sum(v[0] for kk, v in pr.items() if kk.startswith("gemm")) / args.steps
        fl = 2.0 * m * n * k
        gbs = 8.0 * m * n / (ms * 1e-3) / 1e9
        out[name] = dict(ms=ms, tflops=fl / (ms * 1e-3) / 1e12, c_stream_gbs=gbs, hbm_frac=gbs / pk["hbm"])
    head = out["tma_tf32_split"]
    roof = dict(kernel="gemm_tma", bound="hbm", achieved=head["c_stream_gbs"], peak=pk["hbm"], unit="GB/s",
                frac=head["hbm_frac"], traffic=profiled_traffic("gemm_tma"), tflops=head["tflops"],
                tf32_peak_tflops=pk["bf16"] * TF32_PER_BF16,
                note="C += A B with K = 256: 64 flop per byte of the C stream, below the TF32 ridge: HBM bounds it")
    return dict(metric="GEMM of the block update, TFLOP/s (FP32 via TF32 split)", value=head["tflops"],
                unit="TFLOP/s", n_gpus=world, steps=args.steps, warmup=args.warmup, ms_per_step=head["ms"],
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32 (tf32 hi/lo split)",
                data="synthetic", config=dict(workload="gemm_update_8192x8192_k256", m=m, n=n, k=k, beta=1.0,
                                              l2="C (256 MB) exceeds L2"),
                engines=out, roofline=roof, gpu_launches=1)


def cpu_baseline_large(args, res):
    """CPU baseline of the large configurations, where one full-size oracle
    solve would run far beyond the bench's few minutes: the oracle as it stands on the same family at a
    reduced size (64 x 64 p = 3 Helmholtz, 16^3 p = 1
    diffusion with one right-hand side), timed, plus the GPU headline form on
    that same problem against the oracle (apply and solution); the full-size
    check is the true FP64 residual of every solution in the bench line."""
    import oracle
    import torch
    from paper_1508_07798_gb300 import hssnd
    from paper_1508_07798_gb300 import dg_inputs as dg
    spec = dict(LARGE[args.workload])
    n_s, p_s = spec["small"]
    spec["nrhs"] = 1
    mesh, A, b, meshdesc, c_elem, kappa_h = large_problem(spec, 0, n_s, p_s)
    b = b[:, 0]
    Acsr = dg.bsr_to_csr(A)
    t0 = time.perf_counter()
    nd = oracle.nd_order(spec["dim"], mesh.n, p_s, A.row_ptr, A.col_idx, leaf_max=64)
    fac = oracle.factor(Acsr, nd, tol=spec["tol"], seed=0, rmax=spec["rmax"])
    xo, info = oracle.fgmres(lambda v: Acsr @ v, lambda v: oracle.apply(fac, v), b, rtol=RTOL, restart=RESTART)
    dt = time.perf_counter() - t0
    # the GPU forms on the same small problem, against the oracle
    dA = hssnd.DeviceBSR.from_host(A)
    tree = hssnd.nd_order(meshdesc, dA)
    X = dg.random_rhs(A.n, 2, 7)
    errs = {}
    for form in ("fp64", "fp32"):
        F = hssnd.hss_factor(dA, tree, tol=spec["tol"], precision=form, rmax=spec["rmax"],
                             tensor_cores=args.tensor_cores if form == "fp32" else 0,
                             sample_bf16=(spec["bf16"] if args.sample_bf16 is None else args.sample_bf16)
                             if form == "fp32" else 0)
        Y = hssnd.hss_apply(F, torch.as_tensor(X, device="cuda")).cpu().numpy()
        Yo = oracle.apply(fac, X)
        x, st = hssnd.fgmres_solve(dA, F, torch.as_tensor(b, device="cuda"), rtol=RTOL, restart=RESTART)
        errs[form] = dict(apply_rel_err=float(np.linalg.norm(Y - Yo) / np.linalg.norm(Yo)),
                          solution_rel_diff=float(np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)),
                          iters=st.iters, oracle_iters=info["iters"])
    return dict(value=dt * 1e3, unit="ms", cores=cpu_cores(), blas_threads=blas_threads(), kind="oracle",
                sample=f"one {A.n}-dof solve of the same family ({n_s}^{spec['dim']} elements, p={p_s}), "
                       "a reduced size of the same family (a full-size oracle solve would run far beyond the bench's minutes)",
                iters=info["iters"], gpu_vs_oracle_at_sample=errs)


BATCH_COUNT, BATCH_RHS, BATCH_TOL = 256, 32, 1e-6


def bench_batched(args, rank, world):
    """256 independent instances (meshes 16..64 per side, p in {1,2,3}, Poisson
    or Helmholtz drawn per instance), 32 N(0,1) right-hand sides each, FP32
    factors, FP64 FGMRES to 1e-8.  One step = nd_order_batched +
    hss_factor_batched + fgmres_solve_batched for each block-size group."""
    import numpy as np
    import torch
    from paper_1508_07798_gb300 import hssnd
    from paper_1508_07798_gb300 import dg_inputs as dg

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    inst = dg.batched_instances(BATCH_COUNT, master_seed=rank)
    groups = {}
    for d in inst:
        groups.setdefault(d["mesh"].p, []).append(d)
    G = []
    for p, ds in sorted(groups.items()):
        dAs = [hssnd.DeviceBSR.from_host(d["A"]) for d in ds]
        meshes = [(2, (d["mesh"].n[0], d["mesh"].n[1]), p) for d in ds]
        N = sum(A.n for A in dAs)
        Bh = dg.random_rhs(N, BATCH_RHS, 1000 * rank + p, kind="normal")
        G.append(dict(p=p, ds=ds, dAs=dAs, meshes=meshes, N=N, Bh=Bh, B=torch.as_tensor(Bh, device=dev)))
    dofs = sum(g["N"] for g in G)

    def step():
        out = []
        for g in G:
            forest = hssnd.nd_order_batched(g["meshes"], g["dAs"])
            F = hssnd.hss_factor_batched(g["dAs"], forest, tol=BATCH_TOL, precision="fp32", autotune=1)
            X, st = hssnd.fgmres_solve_batched(F, g["B"], rtol=RTOL, restart=RESTART)
            out.append((forest, F, X, st))
        return out

    def timed(n):
        ts, last = [], None
        for _ in range(n):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            last = step()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return ts, last

    for _ in range(args.warmup):
        step()
    clk = Clocks(dev.index)
    clk.start()
    l0 = hssnd.launch_count()
    times, last = timed(args.steps)
    launches = (hssnd.launch_count() - l0) // args.steps
    clocks = clk.stop()
    hssnd.profile_reset()
    hssnd.profile_enable(True)
    timed(1)
    hssnd.profile_enable(False)
    prof = hssnd.profile_read()
    # true residuals of every (instance, rhs) on the CPU, per-group statistics
    worst, conv, iters, groups_out = 0.0, True, [], []
    for g, (forest, F, X, st) in zip(G, last):
        off = forest.inst_dof
        Xh = X.cpu().numpy()
        for i, d in enumerate(g["ds"]):
            Acsr = dg.bsr_to_csr(d["A"])
            bi, xi = g["Bh"][off[i]:off[i + 1]], Xh[off[i]:off[i + 1]]
            worst = max(worst, float((np.linalg.norm(bi - Acsr @ xi, axis=0) / np.linalg.norm(bi, axis=0)).max()))
        conv = conv and all(s_.converged for s_ in st)
        iters += [s_.max_iters for s_ in st]
        info = F.info()
        groups_out.append(dict(p=g["p"], instances=len(g["ds"]), dofs=g["N"], factor_bytes=info["factor_bytes"],
                               front_flops=info["front_flops"], capped_fronts=info["capped_fronts"],
                               max_rank=info["max_rank"]))
    # the same instances one at a time through the single-instance calls, once
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for g in G:
        off = np.concatenate([[0], np.cumsum([A.n for A in g["dAs"]])])
        for i, (A, m) in enumerate(zip(g["dAs"], g["meshes"])):
            t = hssnd.nd_order(m, A)
            F = hssnd.hss_factor(A, t, tol=BATCH_TOL, precision="fp32", autotune=1)
            hssnd.fgmres_solve(A, F, g["B"][off[i]:off[i + 1]], rtol=RTOL, restart=RESTART)
    e1.record(stream)
    torch.cuda.synchronize()
    sequential_ms = e0.elapsed_time(e1)
    # e2e: host copies of every matrix and right-hand side in, solutions out
    pinned = []
    h2d = d2h = 0
    for g in G:
        for d in g["ds"]:
            A = d["A"]
            for arr in (A.row_ptr, A.col_idx, A.val.reshape(-1)):
                t = torch.as_tensor(arr).pin_memory()
                pinned.append((t, torch.empty_like(t, device=dev)))
                h2d += t.numel() * t.element_size()
        bt = torch.as_tensor(g["Bh"]).pin_memory()
        pinned.append((bt, torch.empty_like(bt, device=dev)))
        h2d += bt.numel() * 8
        d2h += bt.numel() * 8
    xh = [torch.empty(g["Bh"].shape, dtype=torch.float64).pin_memory() for g in G]
    ets = []
    for it in range(1 + args.steps):
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for hsrc, ddst in pinned:
            ddst.copy_(hsrc, non_blocking=True)
        out = step()
        for k, (_, _, X, _) in enumerate(out):
            xh[k].copy_(X, non_blocking=True)
        a1.record(stream)
        torch.cuda.synchronize()
        if it >= 1:
            ets.append(a0.elapsed_time(a1))
    kernels = {k: dict(ms=round(v[0], 3), launches=v[1]) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])}
    tracked = {k: v for k, v in prof.items() if v[2] > 0}
    dom = max(tracked, key=lambda k: tracked[k][0])
    pk = with_simt_peak(peaks(), device_sms(dev))
    roof = roofline_of(dom, *prof[dom], sum(v[0] for v in prof.values()), pk)
    value = statistics.mean(times)
    e2e_v = statistics.mean(ets)
    if world > 1:
        value, e2e_v = max_over_ranks([value, e2e_v], dev)
    return dict(metric=METRIC, value=value, unit="ms", n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=value, higher_is_better=False, scaling="weak", vs_baseline=None,
                dtype="f32 factor / f64 Krylov", data="synthetic",
                config=dict(workload="batched_256_instances_32rhs", instances=BATCH_COUNT, rhs=BATCH_RHS, dofs=dofs,
                            id_tol=BATCH_TOL, rtol=RTOL, restart=RESTART, groups=groups_out,
                            l2="inputs larger than L2 (A and the Krylov blocks take tens of GB)",
                            apply_autotune="per-level work split timed in the warm-up, cached for the process",
                            parallelism=f"replicas x{world} (independent batches)"),
                converged=bool(conv and worst <= RTOL * 1.0001), worst_true_relres=worst,
                max_iters=max(iters), sequential_ms=sequential_ms,
                roofline=roof, e2e=dict(value=e2e_v, unit="ms", h2d_bytes_per_step=int(h2d),
                                        d2h_bytes_per_step=int(d2h)),
                clocks=clocks, gpu_launches=int(launches), kernels_instrumented_step=kernels)


def headline_config(args, world):
    """Configuration of the default workload, the same dictionary in both arms
    of the bench (the GPU line and the oracle's reference line)."""
    return dict(workload=WORKLOAD, dofs=N_ELEM * N_ELEM * (P_DEG + 1) ** 2, p=P_DEG, mesh=f"{N_ELEM}x{N_ELEM}",
                id_tol=TOL, rtol=RTOL, restart=RESTART, leaf_max=64, headline_form=args.forms.split(",")[0],
                learned_probe_vectors=args.probe, tensor_cores=args.tensor_cores,
                sample_bf16=args.sample_bf16 or 0,
                l2="flushed by a 256 MB write before every timed step",
                apply_autotune="per-level work split timed on the first factorization of the "
                               "structure (a warm-up step), cached for the process",
                parallelism=f"replicas x{world} (independent instances)")


def cpu_baseline_run(seed=0):
    """The oracle, as it stands, on one full problem of the workload."""
    import numpy as np
    import oracle
    from paper_1508_07798_gb300 import dg_inputs as dg
    mesh, A, b = make_problem(seed)
    Acsr = dg.bsr_to_csr(A)
    t0 = time.perf_counter()
    nd = oracle.nd_order(2, mesh.n, P_DEG, A.row_ptr, A.col_idx, leaf_max=64)
    fac = oracle.factor(Acsr, nd, tol=TOL, seed=0, rmax=96)
    x, info = oracle.fgmres(lambda v: Acsr @ v, lambda v: oracle.apply(fac, v), b, rtol=RTOL, restart=RESTART)
    dt = time.perf_counter() - t0
    return dt * 1e3, info


def cpu_cores():
    """Host cores this process may run on (the oracle's BLAS and NumPy use
    them all)."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        return int(max((d.get("num_threads", 1) for d in threadpool_info()), default=1))
    except Exception:
        return None


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        if rank != 0:
            return
        # the reference arm is the CPU oracle (no reference implementation
        # exists); it keeps no state between solves, so there is nothing to warm
        ts, its = [], None
        for _ in range(args.steps):
            ms, info = cpu_baseline_run(0)
            ts.append(ms)
            its = info["iters"]
        v = statistics.mean(ts)
        line = dict(metric=METRIC, value=v, unit="ms", n_gpus=world, steps=args.steps, warmup=args.warmup,
                    ms_per_step=v, higher_is_better=False, scaling="weak", vs_baseline=None, dtype="f64",
                    data="synthetic", impl="reference",
                    config=headline_config(args, world),
                    cpu_baseline=dict(kind="oracle", cores=cpu_cores(), blas_threads=blas_threads(), value=v,
                                      unit="ms",
                                      sample="one full 36,864-dof solve per step (nd + factor + FGMRES), "
                                             "warm-up skipped (no state to warm)", iters=its),
                    e2e=dict(value=v, unit="ms", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
        print(json.dumps(line))
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build()
    if args.workload == "gemm_update":
        if rank == 0:
            print(json.dumps(bench_gemm_update(args, rank, world)))
        return
    if args.workload in LARGE:
        res = bench_large(args, rank, world)
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            res["cpu_baseline"] = cpu_baseline_large(args, res)
        if rank == 0:
            print(json.dumps(res))
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
            dist.destroy_process_group()
        return
    if args.workload == "batched256":
        res = bench_batched(args, rank, world)
        if rank == 0:
            print(json.dumps(res))
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
            dist.destroy_process_group()
        return
    res = bench_ours(args, rank, world)
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.quick:
        ms, info = cpu_baseline_run(0)
        res["cpu_baseline"] = dict(value=ms, unit="ms", cores=cpu_cores(), blas_threads=blas_threads(), kind="oracle",
                                   sample="one full 36,864-dof solve (nd + factor + FGMRES), seed 0",
                                   iters=info["iters"])
    if rank == 0:
        print(json.dumps(res))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
