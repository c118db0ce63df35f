#!/usr/bin/env python
"""Throughput benchmark of the matrix-valued quantum LBM step on GB300.

Default workload: D3Q19 128^3 periodic, tau = 0.7, beta0 = 1, density,
velocity (|u| <= 0.05) and spin fields as seeded Fourier-mode sums with
|k| <= 4, equilibrium-initialised (the 3D FP64/FP32 configuration).  One
"step" is one time step of the whole forward path: the fused
moments + equilibrium + BGK + in-place streaming kernel; the timed region
ends with the FP64 conservation reduction.  Reported:

  value       MLUPS of the FP32-storage step (sites x steps / s / 1e6)
  roofline    the step kernel's algorithmic bytes (b*4 values read + written
              per site) / its CUDA-event duration, against the measured HBM
              copy bandwidth
  fp64        the same for FP64 storage
  df64        the same for double-float storage (two floats per value,
              double-float arithmetic on the FP32 pipes)
  fp64df      the same for FP64 storage stepped in double-float arithmetic
  e2e         MLUPS through the C ABI with host buffers: init from pinned
              host fields, K steps, moments back to pinned host memory
  adjoint     reverse sweep time (segment recomputation + adjoint steps) /
              plain forward time over the same 256 steps, FP32
  cpu_baseline  the FP64 oracle on a 32^3 sample on the host cores

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs an independent replica (the path has
no exchange step in this build); value = all ranks' site updates / max time.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS and % of HBM roofline (FP64 vs FP32 storage), adjoint/forward time ratio"

WORKLOADS = {
    "d3q19-128": dict(d=3, dims=(128, 128, 128), tau=0.7, beta0=1.0, kind="modes", seed=2,
                      desc="D3Q19 128^3 periodic, tau=0.7, beta0=1, Fourier-mode density/velocity/spin "
                           "fields |k|<=4 (RMS 0.02, |u|<=0.05), equilibrium init, eps=eps0"),
    "d2q9-64": dict(d=2, dims=(64, 64, 1), tau=0.8, beta0=1.0, kind="blob", seed=1,
                    desc="D2Q9 64^2 periodic, tau=0.8, beta0=1, density 1+0.05 sin(2 pi x/64), Gaussian "
                         "spin blob sigma=8 (|r|=0.1 n, seeded Bloch axis), u=0, eps=eps0"),
    "d3q19-512": dict(d=3, dims=(512, 512, 512), tau=0.6, beta0=1.0, kind="modes", seed=5,
                      desc="D3Q19 512^3 periodic, tau=0.6, beta0=1, Fourier-mode fields amplitude 0.02"),
    "d2q9-4096": dict(d=2, dims=(4096, 4096, 1), tau=0.7, beta0=1.0, kind="shear", seed=3,
                      desc="D2Q9 4096^2 periodic double shear layer, opposite spin bands"),
}


def bytes_per_value(prec):
    return {"fp64": 8, "df64": 8, "fp64df": 8, "fp32": 4, "fp16dev": 2}[prec]


def make_fields(w):
    from paper_1309_1656_gb300 import fields
    if w["kind"] == "modes":
        return fields.modes(w["d"], w["dims"], seed=w["seed"])
    if w["kind"] == "shear":
        return fields.shear2d(w["dims"][0], w["dims"][1], seed=w["seed"])
    if w["kind"] == "blob":
        return fields.blob2d(w["dims"][0], w["dims"][1], seed=w["seed"])
    raise ValueError(w["kind"])


STEP_KERNEL_SOURCES = ("lattice.cuh", "step.cuh")


def kernel_source_hash(files=STEP_KERNEL_SOURCES):
    """Hash of the sources that define the step kernel (collision + AA
    addressing); a recorded DRAM traffic is used only while it matches."""
    h = hashlib.sha256()
    for name in files:
        with open(os.path.join(ROOT, "paper_1309_1656_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def recorded_traffic(kernel_key):
    """DRAM bytes per site of a kernel from the committed ncu summary, if it
    was taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(kernel_key)
    if not e or e.get("source_hash") != kernel_source_hash():
        return None
    return float(e["dram_bytes_per_site"])


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_id):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", dev_id, "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) != 7:
                    continue
                try:
                    rows.append((float(parts[0]), float(parts[1]), parts[3:]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_device(lat, K, W, stream, torch):
    """W warm-up steps, then K timed steps + the conservation reduction.
    Returns (step_ms_avg, total_ms)."""
    lat.step(W)
    lat.sync()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e2 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat.step(K)
    e1.record(stream)
    cons = lat.conserved()
    e2.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / K, e0.elapsed_time(e2), cons


def max_over_ranks_of(x, ws, device):
    """The largest of every rank's x (the job's time is its slowest rank's)."""
    if ws == 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_mlups(ws, sites_per_rank, steps, seconds):
    """Whole-job throughput: all ranks' site updates over the slowest time."""
    return ws * sites_per_rank * steps / seconds / 1e6


def bench_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    import __graft_entry__
    from paper_1309_1656_gb300 import _build
    if not _build.up_to_date():
        if rank == 0:
            __graft_entry__.build()
        if ws > 1:
            torch.distributed.barrier()
    from paper_1309_1656_gb300 import qlbm

    w = WORKLOADS[args.workload]
    d, dims = w["d"], w["dims"]
    N = dims[0] * dims[1] * dims[2]
    b = 9 if d == 2 else 19
    K, W = args.steps, args.warmup
    fl = make_fields(w)
    peak, peak_src = measured_peaks()
    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream()
    props = torch.cuda.get_device_properties(dev)
    uuid = str(getattr(props, "uuid", "")) or str(dev)
    dev_id = uuid if uuid.startswith("GPU-") else ("GPU-" + uuid if len(uuid) > 30 else str(dev))

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    def max_over_ranks(x):
        return max_over_ranks_of(x, ws, "cuda")

    results = {}
    clocks = None
    for prec in args.precisions.split(","):
        lat = qlbm.Lattice(d, dims, w["tau"], w["beta0"], precision=prec, stream=stream.cuda_stream)
        lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        c0 = lat.conserved()
        barrier()
        sampler = ClockSampler(dev_id) if prec == "fp32" else None
        step_ms, total_ms, c1 = run_device(lat, K, W, stream, torch)
        if sampler is not None:
            clocks = sampler.stop()
        step_ms = max_over_ranks(step_ms)
        total_ms = max_over_ranks(total_ms)
        alg_bytes = N * b * 4 * 2 * bytes_per_value(prec)
        achieved = alg_bytes / (step_ms * 1e-3) / 1e9
        drift = float(np.max(np.abs(c1 - c0)) / np.max(np.abs(c0)))
        results[prec] = dict(step_ms=step_ms, total_ms=total_ms, achieved=achieved,
                             mlups=job_mlups(ws, N, K, total_ms * 1e-3),
                             kernel_mlups=job_mlups(ws, N, 1, step_ms * 1e-3), drift=drift,
                             alg_bytes=alg_bytes)
        lat.close()
        del lat
        torch.cuda.synchronize()

    # reverse mode: checkpointed rollout + adjoint sweep vs a plain forward
    adj = None
    if "fp32" in results and args.adjoint_steps > 0:
        NA = args.adjoint_steps
        lat = qlbm.Lattice(d, dims, w["tau"], w["beta0"], precision="fp32", stream=stream.cuda_stream)
        lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        lat.step(W)
        lat.sync()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        ev[0].record(stream)
        lat.step(NA)
        ev[1].record(stream)
        lat.sync()
        # an untimed rollout first allocates the checkpoint memory
        lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        qlbm.qlbm_rollout(lat.h, NA, 0)
        lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        torch.cuda.synchronize()
        ev[2].record(stream)
        qlbm.qlbm_rollout(lat.h, NA, 0)
        ev[3].record(stream)
        interval = qlbm.qlbm_rollout_interval(lat.h)
        # observable: total spin magnetisation s_z in the central (L/4)^d box
        lam_T = torch.zeros((b, 4, N), dtype=torch.float64, device="cuda")
        grid = np.zeros(dims[::-1], bool)
        sl = tuple(slice(n // 2 - max(1, n // 8), n // 2 + max(1, n // 8)) for n in dims[::-1])
        grid[sl] = True
        lam_T[:, 3, torch.from_numpy(grid.ravel()).cuda()] = 1.0
        lam_0 = torch.empty_like(lam_T)
        torch.cuda.synchronize()
        ev[4].record(stream)
        dJdtau = qlbm.qlbm_rollout_adjoint(lat.h, lam_T, lam_0)
        ev[5].record(stream)
        torch.cuda.synchronize()
        t_plain = ev[0].elapsed_time(ev[1])
        t_roll = ev[2].elapsed_time(ev[3])
        t_adj = ev[4].elapsed_time(ev[5])
        t_plain = max_over_ranks(t_plain)
        t_roll = max_over_ranks(t_roll)
        t_adj = max_over_ranks(t_adj)
        # the same with square-root checkpointing forced
        ksq = 1
        while ksq * ksq < NA:
            ksq += 1
        lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        qlbm.qlbm_rollout(lat.h, NA, ksq)
        lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        torch.cuda.synchronize()
        ev[2].record(stream)
        qlbm.qlbm_rollout(lat.h, NA, ksq)
        ev[3].record(stream)
        torch.cuda.synchronize()
        ev[4].record(stream)
        dJdtau_sq = qlbm.qlbm_rollout_adjoint(lat.h, lam_T, lam_0)
        ev[5].record(stream)
        torch.cuda.synchronize()
        t_roll_sq = max_over_ranks(ev[2].elapsed_time(ev[3]))
        t_adj_sq = max_over_ranks(ev[4].elapsed_time(ev[5]))
        adj = {"ratio": round(t_adj / t_plain, 3), "unit": "adjoint sweep time / forward time",
               "forward_ms": round(t_plain, 3), "rollout_ms": round(t_roll, 3),
               "adjoint_ms": round(t_adj, 3), "rollout_overhead": round(t_roll / t_plain, 3),
               "steps": NA, "interval": interval, "precision": "fp32",
               "observable": "sum of s_z over the central box", "dJ_dtau": dJdtau,
               "note": "checkpoint interval chosen by the library (1 = every state kept, written by "
                       "the forward steps; the sweep recomputes nothing)",
               "sqrt_checkpoints": {"interval": ksq, "ratio": round(t_adj_sq / t_plain, 3),
                                    "rollout_overhead": round(t_roll_sq / t_plain, 3),
                                    "adjoint_ms": round(t_adj_sq, 3),
                                    "dJ_dtau_matches": dJdtau_sq == dJdtau,
                                    "note": "segment recomputation (two-buffer forward) + reverse steps"}}
        lat.close()
        del lat, lam_T, lam_0
        torch.cuda.synchronize()

    # Fermi-Dirac parameter recovery (side output, FP64 solve) and the FP64
    # step variant whose equilibrium goes through the recovered parameters
    fdp = None
    if args.fd_params and rank == 0:
        lat = qlbm.Lattice(d, dims, w["tau"], w["beta0"], precision="fp64", stream=stream.cuda_stream)
        lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        lat.step(4)
        outs = [torch.empty((N,), dtype=torch.float64, device="cuda") for _ in range(3)]
        ax = torch.empty((3, N), dtype=torch.float64, device="cuda")
        qlbm.qlbm_fd_params(lat.h, *outs, ax)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        nfail = qlbm.qlbm_fd_params(lat.h, *outs, ax)
        ev[1].record(stream)
        lat.set_equilibrium_path(qlbm.QLBM_EQ_FD_PARAMS)
        ns = 10
        lat.step(2)
        lat.sync()
        ev[2].record(stream)
        lat.step(ns)
        ev[3].record(stream)
        torch.cuda.synchronize()
        t_fd = ev[0].elapsed_time(ev[1])
        t_step = ev[2].elapsed_time(ev[3]) / ns
        fdp = {"fd_params_ms": round(t_fd, 3), "fd_params_msites_per_s": round(N / t_fd / 1e3, 1),
               "fd_path_step_ms": round(t_step, 3), "fd_path_mlups": round(N / t_step / 1e3, 1),
               "unresolved_sites": nfail, "beta_median": float(outs[0].median()),
               "note": "FP64 per-site eigen-decomposition + Newton on the 3x3 logarithmic system (Prop. 1); cost reported "
                       "separately, the paper's step does not need it"}
        lat.close()
        del outs, ax
        torch.cuda.synchronize()
        # the FP32 step with the single-precision solve fused in: every step
        # also writes (beta, mu_up, mu_dn, axis) as float [6][N]
        if "fp32" in results:
            lat = qlbm.Lattice(d, dims, w["tau"], w["beta0"], precision="fp32", stream=stream.cuda_stream)
            lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
            o32 = [torch.empty((N,), dtype=torch.float32, device="cuda") for _ in range(3)]
            a32 = torch.empty((3, N), dtype=torch.float32, device="cuda")
            for _ in range(W):
                qlbm.qlbm_step_fd_output(lat.h, *o32, a32, count=False)
            lat.sync()
            torch.cuda.synchronize()
            nf = 100
            ev[0].record(stream)
            for _ in range(nf):
                qlbm.qlbm_step_fd_output(lat.h, *o32, a32, count=False)
            ev[1].record(stream)
            torch.cuda.synchronize()
            t_f = ev[0].elapsed_time(ev[1]) / nf
            nfail32 = qlbm.qlbm_step_fd_output(lat.h, *o32, a32)
            fbytes = N * (b * 4 * 2 * 4 + 6 * 4)
            fdp["fused_fp32"] = {
                "step_ms": round(t_f, 4), "mlups": round(N / t_f / 1e3, 1),
                "vs_plain_step": round(t_f / results["fp32"]["step_ms"], 3),
                "achieved_gbs": round(fbytes / (t_f * 1e-3) / 1e9, 1),
                "hbm_frac": round(fbytes / (t_f * 1e-3) / 1e9 / peak, 4),
                "bytes_per_site": b * 4 * 2 * 4 + 6 * 4, "unresolved_sites": nfail32,
                "note": "FP32 step + per-site single-precision FD solve (double where the float "
                        "iteration does not settle), parameters written every step"}
            lat.close()
            del o32, a32
            torch.cuda.synchronize()

    # end-to-end through the C ABI with pinned host buffers
    e2e = None
    if "fp32" in results and not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        r4, uu = pin(fl["rho4"]), pin(fl["u"])
        out_r = torch.empty((4, N), dtype=torch.float64).pin_memory().numpy()
        out_u = torch.empty((d, N), dtype=torch.float64).pin_memory().numpy()
        out_e = torch.empty((N,), dtype=torch.float64).pin_memory().numpy()
        lat = qlbm.Lattice(d, dims, w["tau"], w["beta0"], precision="fp32", stream=stream.cuda_stream)
        lat.init_equilibrium(r4, uu)       # warm the staging buffers
        lat.step(W)
        qlbm.qlbm_moments(lat.h, out_r, out_u, out_e)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        qlbm.qlbm_init_equilibrium(lat.h, r4, uu, None)
        qlbm.qlbm_step(lat.h, K)
        qlbm.qlbm_moments(lat.h, out_r, out_u, out_e)
        t1 = time.perf_counter()
        dt_e2e = max_over_ranks(t1 - t0)
        lat.close()
        e2e = {"value": round(job_mlups(ws, N, K, dt_e2e), 3), "unit": "MLUPS",
               "h2d_bytes_per_step": (r4.nbytes + uu.nbytes) / K,
               "d2h_bytes_per_step": (out_r.nbytes + out_u.nbytes + out_e.nbytes) / K}

    growth = None
    if args.error_growth > 0 and rank == 0:
        growth = error_growth(w, fl, args.error_growth, args.error_every, torch, qlbm)

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    def parity(sdims, sfl, nsteps, st_ref, mom_ref):
        """Errors of the GPU precisions against the oracle on the CPU sample
        (normwise, max |x - x_ref| / max |x_ref|)."""
        err = lambda a, b_: float(np.max(np.abs(a - b_)) / np.max(np.abs(b_)))
        res = {"steps": nsteps, "norm": "max |x - x_oracle| / max |x_oracle|"}
        for prec in ("fp64", "fp64df", "df64", "fp32", "fp16dev"):
            with qlbm.Lattice(d, sdims, w["tau"], w["beta0"], precision=prec) as lat:
                lat.init_equilibrium(sfl["rho4"], sfl["u"], sfl["eps"])
                lat.step(nsteps)
                r4, uu, ee = lat.moments()
                e = {"n": err(r4[0], mom_ref[0][0]), "S": err(r4[1:], mom_ref[0][1:]),
                     "u": err(uu, mom_ref[1]), "eps": err(ee, mom_ref[2])}
                if prec in ("fp64", "fp64df", "df64"):
                    e["state"] = err(lat.get_state(), st_ref)
                    e["state_per_step"] = e["state"] / nsteps
                res[prec] = {k: float("%.3g" % v) for k, v in e.items()}
        return res

    cpu = None
    if ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(w, target_s=args.cpu_seconds, parity_fn=parity)

    r32 = results.get("fp32") or next(iter(results.values()))
    prim = "fp32" if "fp32" in results else next(iter(results))
    traffic = recorded_traffic("step_%s_d%d" % (prim, d))
    roof = {"bound": "hbm", "achieved": round(r32["achieved"], 1), "peak": peak, "unit": "GB/s",
            "frac": round(r32["achieved"] / peak, 4), "peak_source": peak_src,
            "traffic": None if traffic is None else round(traffic * N),
            "algorithmic_bytes_per_launch": r32["alg_bytes"],
            "kernel": "k_step_aa<%d,%s>" % (d, prim)}
    if traffic is not None:
        # DRAM bytes actually moved per launch (ncu) over the same event time:
        # below the algorithmic bytes by the writes still in L2 at kernel end
        dram = traffic * N / (r32["step_ms"] * 1e-3) / 1e9
        roof["dram_achieved"] = round(dram, 1)
        roof["dram_frac"] = round(dram / peak, 4)
    line = {
        "metric": METRIC, "value": round(r32["mlups"], 1), "unit": "MLUPS", "n_gpus": ws,
        "steps": K, "warmup": W, "ms_per_step": round(r32["total_ms"] / K, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "fp16dev": "f16-storage/f32", "df64": "f32x2",
                  "fp64df": "f64-storage/f32x2"}[prim],
        "data": "synthetic",
        "config": {"workload": w["desc"], "lattice": "D3Q19" if d == 3 else "D2Q9",
                   "dims": list(dims), "sites": N, "tau": w["tau"], "beta0": w["beta0"],
                   "precision": prim, "parallelism": "replicas" if ws > 1 else "single-gpu",
                   "l2": ("inputs larger than L2: state %.2f GB > 129 MB, no flush" if
                          N * b * 4 * bytes_per_value(prim) > 129e6 else
                          "state %.4f GB fits in the 129 MB L2: L2-resident by construction, "
                          "not an HBM measurement") % (N * b * 4 * bytes_per_value(prim) / 1e9)},
        "roofline": roof,
        "kernel_mlups": round(r32["kernel_mlups"], 1),
        "conservation_drift_rel": r32["drift"],
        "gpu_launches": K + 2,
    }
    for p_, r in results.items():
        if p_ == prim:
            continue
        line[p_] = {"value": round(r["mlups"], 1), "unit": "MLUPS",
                    "kernel_mlups": round(r["kernel_mlups"], 1),
                    "achieved_gbs": round(r["achieved"], 1), "hbm_frac": round(r["achieved"] / peak, 4),
                    "conservation_drift_rel": r["drift"]}
        if p_ == "fp64":
            # bound by FP64 issue: 2 FP64 lanes/clk/SM x 152 SMs x clock
            line[p_]["bound"] = "alu (fp64 pipe, see profiles/k_step_aa_d3q19_fp64_128.md)"
        if p_ == "fp64df":
            line[p_]["bound"] = ("alu (fp64 pipe: moment sums and rounding; integer pipe: splits; see "
                                 "profiles/k_step_aa_f64df_d3q19_fp64df_128.md)")
    if growth:
        line["error_growth"] = growth
    if clocks:
        line["clocks"] = clocks
    if e2e:
        line["e2e"] = e2e
    if adj:
        line["adjoint"] = adj
    if fdp:
        line["fd_params"] = fdp
    if cpu:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def error_growth(w, fl, total, every, torch, qlbm):
    """Normwise errors of the double-float, FP32 and FP16-deviation moment
    fields against the FP64 run of the same workload, every `every` steps."""
    d, dims = w["d"], w["dims"]
    N = dims[0] * dims[1] * dims[2]
    lats = {p: qlbm.Lattice(d, dims, w["tau"], w["beta0"], precision=p) for p in ("fp64", "df64", "fp32", "fp16dev")}
    for lat in lats.values():
        lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
    bufs = {p: (torch.empty((4, N), dtype=torch.float64, device="cuda"),
                torch.empty((d, N), dtype=torch.float64, device="cuda"),
                torch.empty((N,), dtype=torch.float64, device="cuda")) for p in lats}
    out = []
    t = 0
    while t < total:
        n = min(every, total - t)
        for lat in lats.values():
            lat.step(n)
        t += n
        for p, lat in lats.items():
            qlbm.qlbm_moments(lat.h, *bufs[p])
        ref = bufs["fp64"]

        def err(a, b_):
            return float((a - b_).abs().max() / b_.abs().max())

        row = {"step": t}
        for p in ("df64", "fp32", "fp16dev"):
            r, u, e = bufs[p]
            row[p] = {"n": err(r[0], ref[0][0]), "S": err(r[1:], ref[0][1:]), "u": err(u, ref[1]),
                      "eps": err(e, ref[2])}
        out.append(row)
    for lat in lats.values():
        lat.close()
    return {"reference": "the FP64 GPU run of the same workload (itself within 1e-12/step of the oracle)",
            "norm": "max |x - x_fp64| / max |x_fp64| per field", "rows": out}


def cpu_sample(w, L=32):
    from paper_1309_1656_gb300 import fields
    d = w["d"]
    if w["kind"] == "blob":
        return w["dims"], make_fields(w)
    dims = (L, L, L) if d == 3 else (L * 8, L * 8, 1)
    fl = fields.modes(d, dims, seed=w["seed"]) if w["kind"] == "modes" else \
        fields.shear2d(dims[0], dims[1], seed=w["seed"], delta=max(2.0, 80.0 * dims[1] / 4096.0))
    return dims, fl


def cpu_baseline(w, target_s=15.0, parity_fn=None):
    """The FP64 oracle, as it stands, on a bounded sample of the workload.
    With parity_fn, the GPU precisions run the same sample for 1000 steps
    and report their error against the oracle's result."""
    import oracle
    oracle.build()
    d = w["d"]
    dims, fl = cpu_sample(w)
    N = dims[0] * dims[1] * dims[2]
    cores = oracle.max_threads(0)
    st = oracle.init_equilibrium(d, dims, w["beta0"], fl["rho4"], fl["u"], fl["eps"])
    st = oracle.run(d, dims, w["tau"], w["beta0"], 2, st)      # thread start-up
    # run in chunks until the sample has taken target_s of wall time
    n, chunk, dt = 0, 8, 0.0
    while dt < target_s:
        t = time.perf_counter()
        st = oracle.run(d, dims, w["tau"], w["beta0"], chunk, st)
        dt += time.perf_counter() - t
        n += chunk
        chunk = min(2 * chunk, 4096)
    out = {"value": round(N * n / dt / 1e6, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
           "sample": "%s sub-lattice %s of the same workload recipe, %d FP64 steps, %.1f s" %
                     ("D3Q19" if d == 3 else "D2Q9", "x".join(map(str, dims)), n, dt)}
    if parity_fn is not None:   # 1000 steps: the fields have not yet relaxed away
        st = oracle.init_equilibrium(d, dims, w["beta0"], fl["rho4"], fl["u"], fl["eps"])
        st = oracle.run(d, dims, w["tau"], w["beta0"], 1000, st)
        out["parity"] = parity_fn(dims, fl, 1000, st, oracle.moments(d, dims, w["beta0"], st))
    return out


def bench_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    w = WORKLOADS[args.workload]
    d = w["d"]
    dims, fl = cpu_sample(w)
    N = dims[0] * dims[1] * dims[2]
    cores = oracle.max_threads(0)
    st = oracle.init_equilibrium(d, dims, w["beta0"], fl["rho4"], fl["u"], fl["eps"])
    st = oracle.run(d, dims, w["tau"], w["beta0"], args.warmup, st)
    t = time.perf_counter()
    oracle.run(d, dims, w["tau"], w["beta0"], args.steps, st)
    dt = time.perf_counter() - t
    v = N * args.steps / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "MLUPS",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt * 1e3 / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["desc"], "sample": "x".join(map(str, dims)),
                       "note": "reference arm = the FP64 CPU oracle (no reference implementation exists)"},
            "cpu_baseline": {"value": round(v, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": "%s sub-lattice %s per step" %
                                       ("D3Q19" if d == 3 else "D2Q9", "x".join(map(str, dims)))},
            "e2e": {"value": round(v, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="d3q19-128", choices=sorted(WORKLOADS))
    ap.add_argument("--precisions", default="fp32,fp64,fp64df,df64")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--adjoint-steps", type=int, default=256)
    ap.add_argument("--error-growth", type=int, default=0,
                    help="also run FP64/FP32/FP16 side by side for this many steps and report errors")
    ap.add_argument("--error-every", type=int, default=1000)
    ap.add_argument("--no-fd-params", dest="fd_params", action="store_false",
                    help="skip timing the Fermi-Dirac parameter recovery")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        bench_reference(args)
    else:
        bench_ours(args)


if __name__ == "__main__":
    main()
