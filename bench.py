#!/usr/bin/env python
"""Benchmark: converged Laplace-domain BEM frequency solves per second on GB300.

Workload (one "step" = one batched solve of every frequency): pressurised spherical cavity in a
full space, icosphere of radius 1 m with 5120 flat triangles (15360 complex unknowns),
mu = 1e9 Pa, nu = 0.25, rho = 2000 kg/m^3, step pressure 1e6 Pa, the 128 frequencies
s_k = 250 + i k pi / 0.02 (k = 0..127), GMRES(50) to ||b - A x|| / ||b|| <= 1e-6 measured in
FP64, FP32 matrix-free operator with FP64 iterative refinement.

value : solves/s with the frequency list, the mesh and the output already in device memory.
e2e   : the same through the C ABI with host buffers (mesh, boundary data and frequencies
        uploaded, all solutions downloaded, every step).
Also reported: the plain-FP64 GPU path on all 128 frequencies; the accuracy of the timed
solutions and of a tol-1.5e-7 solve against a tol-1e-9 one (elementwise and in the FSM transients);
the per-kernel rooflines (executed flops over CUDA-event times of each launch on the launching
stream, against FP32 / FP64 peaks measured in the same run); SM clocks sampled during the timed
region; and the FP64 CPU oracle on a bounded sample (cpu_baseline).

--impl reference times the CPU oracle (dense assembly + LU, FP64) on the same workload: each
step is a bounded sample (a block of matrix rows at one frequency plus an LU of a smaller dense
system), extrapolated to one full solve.
Multi-GPU (torchrun, N ranks): every rank solves its own 128 frequencies of an N*128 frequency
grid (weak scaling, no collective on the data path); value = all solves / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

LEVEL = 4            # 5120 triangles
N_FREQ = 128
T_WIN = 0.02
SIGMA = 250.0
TOL = 1e-6
# Residual tolerance at which the mixed path's solutions meet 1e-6 relative error elementwise
# (against a tol-1e-9 solve of the same discretisation and the oracle's dense LU): a residual of
# 1e-6 ||b|| leaves solution errors up to ~5e-6 max|x| at the top of the band
TOL_ACCURATE = 1.5e-7
TOL_REFERENCE = 1e-9
ACC_ELEMENTS = (0, 700, 1500, 2560, 3333, 4000, 4600, 5119)  # radial displacement responses
METRIC = "BEM frequency solves/s at 1e-6 rel. residual vs plain FP64 GPU; % FP32 peak"
# FP32 far-field kernel, traction columns: FP32 flops per kernel evaluation counted from the
# kernel source (FMA = 2; exp/sin/cos on the special-function unit not counted)
FLOPS_PER_UNIT_T = 159
FLOPS_PER_UNIT_U = 113   # displacement-kernel (U) columns: the right-hand side pass
FLOPS_PER_UNIT_RES = 221  # fused FP64 residual r = K k - A x: T and U per kernel evaluation
# The same residual in float-float on the FP32 pipes (resid_df_kernel, lazily renormalised
# pairs): FP32 flops per kernel evaluation, FADD + FMUL + 2 FFMA thread-instructions of one launch
# (ncu executed-instruction counters, 24 frequencies on 5120 triangles) divided by its units
FLOPS_PER_UNIT_RES_DF = 1537.5  # FADD 749.4 + FMUL 135.3 + 2 x FFMA 326.6 per unit
SMS, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0  # nominal, for the derived-peak note only
# Executed flops per kernel evaluation of the far-field kernels (FADD + FMUL + 2 FFMA, resp.
# DADD + DMUL + 2 DFMA thread instructions from ncu executed-instruction counters divided by the
# launches' units): the FP32 kernel over every far32 launch of one benchmark solve (the mix of
# its recurrence and direct instantiations), the FP64 kernel on the 24-frequency kernel case
FLOPS_EXEC_PER_UNIT_FAR32 = 149.4   # 4.449e13 flop over the 2.978e11 units of one solve's 80 launches
FLOPS_EXEC_PER_UNIT_FAR64 = 287.4   # 7.231e11 flop over the 2.516e9 units of one launch
# DRAM bytes (read + write) of one FP32 far-kernel launch from an ncu capture of the 24-frequency
# kernel case (5120 triangles, 24 x 5120 x 5119 x 4 units): the source vectors, the geometry and
# the FP64 accumulator lines the atomic adds pull in, all proportional to the frequencies (units)
# of a launch, so the roofline scales it to the benchmark's average launch
FAR32_CAPTURE_BYTES, FAR32_CAPTURE_UNITS = 1.00224e7, 24 * 5120 * 5119 * 4


def workload_config(n_gpus):
    return {
        "workload": "pressurised spherical cavity, icosphere 5120 flat triangles (15360 complex "
                    "unknowns), 128 frequencies s_k=250+i*k*pi/0.02, GMRES(50) to 1e-6 FP64 "
                    "residual, FP32 operator + FP64 refinement",
        "n_triangles": 20 * 4 ** LEVEL, "n_unknowns": 3 * 20 * 4 ** LEVEL,
        "n_freq_per_gpu": N_FREQ, "tol": TOL, "restart": 50,
        "l2": "flushed between timed steps (256 MiB device write)",
        "parallelism": f"frequency shards x{n_gpus}" if n_gpus > 1 else "single GPU",
    }


# ------------------------------------------------------------------------------ helpers
class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 7:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for nm, v in zip(names, p[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------------------------ CPU oracle
def oracle_sample(rows=128, n_lu=3072, seed=0):
    """Oracle cost of one full solve of the workload, from a bounded sample: dense assembly of
    `rows` matrix block-rows at one mid-band frequency, and an LU solve of an n_lu dense complex
    system; extrapolated by 5120/rows (assembly) and (15360/n_lu)^3 (LU)."""
    from oracle import bem as OB

    prob = W.spherical_cavity(level=LEVEL, n_freq=N_FREQ, T=T_WIN, sigma=SIGMA)
    g = OB.geometry(prob.verts, prob.tris)
    ne = len(prob.tris)
    sel = np.linspace(0, ne - 1, rows).astype(int)
    t0 = time.perf_counter()
    OB.operators(g, prob.s[64], prob.material, prob.bc_type, rows=sel)
    t_asm = time.perf_counter() - t0
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n_lu, n_lu)) + 1j * rng.standard_normal((n_lu, n_lu))
    b = rng.standard_normal(n_lu) + 0j
    t0 = time.perf_counter()
    np.linalg.solve(A, b)
    t_lu = time.perf_counter() - t0
    per_solve = t_asm * ne / rows + t_lu * (3 * ne / n_lu) ** 3
    sample = (f"dense assembly of {rows} of {ne} block-rows at s_64 ({t_asm:.2f} s, x{ne / rows:.0f}) "
              f"+ LU of a {n_lu}^2 complex system ({t_lu:.2f} s, x{(3 * ne / n_lu) ** 3:.0f}); "
              f"extrapolated {per_solve:.0f} s per solve")
    return 1.0 / per_solve, sample, t_asm + t_lu


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    cores = os.cpu_count()
    for _ in range(args.warmup):
        oracle_sample()
    vals, walls = [], []
    for _ in range(args.steps):
        v, sample, wall = oracle_sample()
        vals.append(v)
        walls.append(wall)
    value = float(np.median(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        # one step is the whole workload (N_FREQ solves), as in the GPU arm; extrapolated from
        # the sample, whose own wall time is sample_wall_s
        "ms_per_step": 1e3 * N_FREQ / value, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.gpus),
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "sample_wall_s": float(np.median(walls)),
        "ms_per_step_note": f"extrapolated time of {N_FREQ} oracle solves (one step of the workload)",
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------ GPU
def run_gpu(args):
    import torch

    import paper_1511_04355_gb300 as P

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.current_stream(dev)

    from paper_1511_04355_gb300 import shard as SH

    prob = W.spherical_cavity(level=LEVEL, n_freq=N_FREQ * ws, T=T_WIN, sigma=SIGMA)
    s_all = SH.shard(prob.s, rank, ws)              # N_FREQ contiguous frequencies per rank
    ne = len(prob.tris)
    n_unk = 3 * ne
    m = prob.material

    ctx = P.Context(local, stream.cuda_stream)
    ctx.set_mesh(prob.verts, prob.tris)
    ctx.set_material(m.mu, m.nu, m.rho)
    ctx.set_bc(prob.bc_type, prob.bc_value, P.BEM_PROFILE_STEP)
    ctx.set_options(precision=P.BEM_PREC_MIXED, tol=TOL)

    s_dev = torch.from_numpy(np.ascontiguousarray(s_all)).to(dev)
    x_dev = torch.zeros((N_FREQ, n_unk), dtype=torch.complex128, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    def step():
        _, info = P.bem_solve_frequencies(ctx.h, s_dev, x_dev)
        return info

    for _ in range(args.warmup):
        flush.zero_()
        step()
    # timed region: device-resident inputs
    launches = 0
    times = []
    infos = []
    ctx.profile(True)
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = step()
            e1.record(stream)
            barrier()
            times.append(e0.elapsed_time(e1))
            launches += int(info["kernel_launches"])
            infos.append(info)
    ktimes = ctx.kernel_times()
    ctx.profile(False)
    t_step = SH.max_over_ranks(float(np.mean(times)), dev)
    value = SH.aggregate_rate(N_FREQ, ws, t_step / 1e3)

    # e2e through the ABI with host buffers (pinned), every step uploads mesh, data, s and
    # downloads all solutions
    verts = np.ascontiguousarray(prob.verts)
    tris = np.ascontiguousarray(prob.tris, dtype=np.int32)
    x_host_t = torch.empty((N_FREQ, n_unk), dtype=torch.complex128, pin_memory=True)
    x_host = x_host_t.numpy()
    s_host = np.ascontiguousarray(s_all)
    h2d = verts.nbytes + tris.nbytes + prob.bc_type.nbytes + prob.bc_value.nbytes + s_host.nbytes
    d2h = x_host.nbytes

    def e2e_step():
        P.bem_set_mesh(ctx.h, verts, tris)
        P.bem_set_material(ctx.h, m.mu, m.nu, m.rho)
        P.bem_set_bc(ctx.h, prob.bc_type, prob.bc_value, P.BEM_PROFILE_STEP)
        P.bem_solve_frequencies(ctx.h, s_host, x_host)

    e2e_step()
    et = []
    for _ in range(args.steps):
        flush.zero_()
        barrier()
        t0 = time.perf_counter()
        e2e_step()
        barrier()
        et.append(time.perf_counter() - t0)
    t_e2e = SH.max_over_ranks(float(np.mean(et)), dev)
    e2e_value = SH.aggregate_rate(N_FREQ, ws, t_e2e)

    def timed_solve(s_d, x_d):
        barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _, inf = P.bem_solve_frequencies(ctx.h, s_d, x_d)
        b.record(stream)
        barrier()
        return a.elapsed_time(b) / 1e3, inf

    # accuracy: the timed solutions, and the mixed path at the tolerance whose solutions meet
    # 1e-6 relative error, against a tol-1e-9 solve of the same discretisation (frequency
    # responses elementwise, radial-displacement time responses by the FSM)
    x_mixed = x_dev.cpu().numpy()
    ctx.set_options(precision=P.BEM_PREC_MIXED, tol=TOL_REFERENCE)
    x_ref_d = torch.zeros_like(x_dev)
    _, info_ref = P.bem_solve_frequencies(ctx.h, s_dev, x_ref_d)
    x_ref = x_ref_d.cpu().numpy()
    ctx.set_options(precision=P.BEM_PREC_MIXED, tol=TOL_ACCURATE)
    x_acc_d = torch.zeros_like(x_dev)
    timed_solve(s_dev, x_acc_d)                     # warm-up at this tolerance
    t_acc, info_acc = timed_solve(s_dev, x_acc_d)
    x_acc = x_acc_d.cpu().numpy()
    nrm = W.unit_normals(prob.verts, prob.tris)
    els = np.array(ACC_ELEMENTS)
    t_out = np.linspace(0.0, 0.01, 200)

    def radial_time(x):
        # outward radial displacement of the cavity wall (normals point into the cavity)
        u = x.reshape(len(x), ne, 3)[:, els, :]
        ur = -np.einsum("fed,ed->fe", u, nrm[els])
        return ctx.fsm_eval(np.ascontiguousarray(ur), SIGMA, 2 * T_WIN, t_out, 1)

    h_ref = radial_time(x_ref)

    def errors(x):
        ew = np.abs(x - x_ref).max(axis=1) / np.abs(x_ref).max(axis=1)
        ht = radial_time(x)
        et = np.abs(ht - h_ref).max(axis=0) / np.abs(h_ref).max(axis=0)
        return float(ew.max()), int(ew.argmax()), float(et.max())

    e_f, k_f, e_t = errors(x_mixed)
    e_fa, k_fa, e_ta = errors(x_acc)

    # the plain-FP64 GPU path (FP64 operator and GMRES) over all frequencies of the step
    ctx.set_options(precision=P.BEM_PREC_FP64, tol=TOL)
    x64 = torch.zeros_like(x_dev)
    P.bem_solve_frequencies(ctx.h, s_dev[:2].contiguous(), x64[:2])   # warm-up of the FP64 path
    ctx.profile(True)
    t64, info64 = timed_solve(s_dev, x64)
    kt64 = ctx.kernel_times()
    ctx.profile(False)
    fp64_value = N_FREQ / t64
    e_f64, _, e_t64 = errors(x64.cpu().numpy())
    ctx.set_options(precision=P.BEM_PREC_MIXED, tol=TOL)

    # measured FP32 and FP64 peaks (FMA-chain kernels, CUDA events), clocks sampled meanwhile
    # (FFMA chains and paired FFMA2 chains: the FP32 peak is the faster of the two)
    with ClockSampler(local) as clk_peak:
        peak32_ffma, _, n_sm = P.bem_measure_peak(ctx.h, P.BEM_PEAK_FP32, 2048, 5)
        peak32_ffma2, _, _ = P.bem_measure_peak(ctx.h, P.BEM_PEAK_FP32X2, 2048, 5)
        peak64, _, _ = P.bem_measure_peak(ctx.h, P.BEM_PEAK_FP64, 512, 5)
    peak32 = max(peak32_ffma, peak32_ffma2)

    if rank != 0:
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel class (device time summed over the timed steps)
    clocks = clk.summary()
    per_step = {k: (n / args.steps, ms / args.steps, fl / args.steps) for k, (n, ms, fl) in ktimes.items()}
    dominant = max(ktimes, key=lambda k: ktimes[k][1])
    info = infos[-1]
    # FP32 far kernel units: every launch covers (ne^2 - ne) x 4 source points x its listed
    # (active) frequencies; the library counts the frequency-launches
    n32, ms32, fl32 = per_step["far32"]
    units32 = fl32 * (ne * ne - ne) * 4
    peak_note = (f"measured: the faster of FFMA- and FFMA2-chain kernels ({peak32_ffma:.1f} / "
                 f"{peak32_ffma2:.1f} TFLOP/s) on {n_sm} SMs, best of 5 launches (CUDA events), "
                 f"SM clock median {clk_peak.summary().get('sm_mhz')} MHz; nominal "
                 f"{n_sm} SMs x {FP32_LANES} lanes x 2 x {SM_MAX_MHZ:.0f} MHz = "
                 f"{n_sm * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12:.1f} TFLOP/s")
    ach32_direct = units32 * FLOPS_PER_UNIT_T / (ms32 / 1e3) / 1e12 if ms32 > 0 else 0.0
    ach32 = units32 * FLOPS_EXEC_PER_UNIT_FAR32 / (ms32 / 1e3) / 1e12 if ms32 > 0 else 0.0
    # FP64-class refinement residual (fused U + T far-field sweep in float-float on the FP32
    # pipes), one launch per full residual
    n64, ms64, fl64 = per_step["res64"]
    flops64 = fl64 * (ne * ne - ne) * 4 * FLOPS_PER_UNIT_RES_DF
    ach64 = flops64 / (ms64 / 1e3) / 1e12 if ms64 > 0 else 0.0
    roof32 = {"kernel": "far32_kernel (FP32 far-field operator)", "bound": "alu",
              "achieved": ach32, "peak": peak32, "unit": "TFLOP/s", "frac": ach32 / peak32,
              "flop_per_unit": FLOPS_EXEC_PER_UNIT_FAR32,
              "flop_count": "executed FP32 flops (ncu FADD + FMUL + 2 FFMA thread instructions per "
                            "kernel evaluation)",
              "achieved_direct_equivalent": ach32_direct,
              "frac_direct_equivalent": ach32_direct / peak32,
              "direct_equivalent_note": f"{FLOPS_PER_UNIT_T} flop per evaluation counted on the direct "
                                        "formulation (what the frequency recurrence and the per-element "
                                        "application avoid computing)",
              "traffic": (FAR32_CAPTURE_BYTES * (units32 / n32) / FAR32_CAPTURE_UNITS
                          if n32 and ne == 5120 else None),
              "traffic_unit": "bytes per launch (ncu 24-frequency capture scaled by units)",
              "launches_per_step": n32, "ms_per_step": ms32, "peak_note": peak_note}
    roof64 = {"kernel": "resid_df_kernel (FP64-class refinement residual r = K k - A x, float-float)",
              "bound": "alu", "achieved": ach64, "peak": peak32, "unit": "TFLOP/s",
              "frac": ach64 / peak32, "traffic": None, "launches_per_step": n64,
              "ms_per_step": ms64, "flop_per_unit": FLOPS_PER_UNIT_RES_DF,
              "flop_count": "executed FP32 flops (ncu FADD + FMUL + 2 FFMA thread instructions per "
                            "kernel evaluation)", "peak_note": peak_note}
    # the plain-FP64 path's far kernel (FP64 operator in its GMRES) against the FP64 peak
    n_f64, ms_f64, fl_f64 = kt64["far64"]
    ach_f64 = (fl_f64 * (ne * ne - ne) * 4 * FLOPS_EXEC_PER_UNIT_FAR64 / (ms_f64 / 1e3) / 1e12
               if ms_f64 > 0 else 0.0)
    roof_fp64 = {"kernel": "far_kernel<double> (FP64 far-field operator of the plain-FP64 path)",
                 "bound": "alu", "achieved": ach_f64, "peak": peak64, "unit": "TFLOP/s",
                 "frac": ach_f64 / peak64, "flop_per_unit": FLOPS_EXEC_PER_UNIT_FAR64,
                 "flop_count": "executed FP64 flops (ncu DADD + DMUL + 2 DFMA thread instructions per "
                               "kernel evaluation)",
                 "launches": n_f64, "ms": ms_f64, "share_of_fp64_path": ms_f64 / 1e3 / t64,
                 "peak_note": "measured: DFMA-chain kernel, best of 5 launches (CUDA events)"}
    roofline = roof64 if dominant == "res64" else roof32

    cpu_v, cpu_sample, _ = (None, None, None)
    if ws == 1 and not args.skip_cpu:
        cpu_v, cpu_sample, _ = oracle_sample()
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic", "config": workload_config(ws),
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": launches,
        "clocks": clocks,
        "roofline": roofline,
        "roofline_fp32_operator": roof32,
        "roofline_residual": roof64,
        "kernel_ms_per_step": {k: v[1] for k, v in per_step.items()},
        "fp64_gpu_path": {"value": fp64_value, "unit": "solves/s", "seconds": t64,
                          "sample": f"all {N_FREQ} frequencies of the step, tol {TOL}",
                          "speedup_mixed_vs_fp64": value / fp64_value,
                          "iterations": info64["iterations"].tolist(),
                          "max_rel_err_elementwise": e_f64, "max_rel_err_time": e_t64,
                          "roofline": roof_fp64},
        "accuracy": {"reference": f"mixed path at tol {TOL_REFERENCE} (max FP64-class residual "
                                  f"{float(np.max(info_ref['residual'])):.2e})",
                     "metric_elementwise": "max_k max_n |x_kn - xref_kn| / max_n |xref_kn|",
                     "metric_time": f"max over t in [0, 10 ms] of |u_r(t) - u_r,ref(t)| / max |u_r,ref| "
                                    f"(FSM of the radial displacement at elements {list(ACC_ELEMENTS)})",
                     "at_tol": {"tol": TOL, "max_fp64_residual": float(np.max(info["residual"])),
                                "max_rel_err_elementwise": e_f, "worst_frequency": k_f,
                                "max_rel_err_time": e_t, "solves_per_s": value,
                                "gmres_iterations": int(np.sum(info["iterations"]))},
                     "at_accurate_tol": {"tol": TOL_ACCURATE,
                                         "max_fp64_residual": float(np.max(info_acc["residual"])),
                                         "max_rel_err_elementwise": e_fa, "worst_frequency": k_fa,
                                         "max_rel_err_time": e_ta,
                                         "solves_per_s": SH.aggregate_rate(N_FREQ, ws, t_acc),
                                         "gmres_iterations": int(np.sum(info_acc["iterations"]))},
                     "iterations": info["iterations"].tolist(),
                     "refinements": info["refinements"].tolist()},
        "peaks_measured": {"fp32_tflops": peak32, "fp32_ffma_tflops": peak32_ffma,
                           "fp32_ffma2_tflops": peak32_ffma2, "fp64_tflops": peak64, "sm_count": n_sm,
                           "clocks": clk_peak.summary()},
    }
    if cpu_v is not None:
        line["cpu_baseline"] = {"value": cpu_v, "unit": "solves/s", "cores": os.cpu_count(),
                                "kind": "oracle", "sample": cpu_sample}
    print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


def kernel_case_single():
    """Small case for ncu captures of a single-frequency FP32 operator launch (the AFS step's
    shape): the 5120-triangle cavity at s_64 alone, one FP32 application after a warm-up."""
    import torch

    import paper_1511_04355_gb300 as P

    prob = W.spherical_cavity(level=LEVEL, n_freq=N_FREQ, T=T_WIN, sigma=SIGMA)
    c = P.Context(0)
    c.set_mesh(prob.verts, prob.tris)
    m = prob.material
    c.set_material(m.mu, m.nu, m.rho)
    c.set_bc(prob.bc_type, prob.bc_value)
    ne = len(prob.tris)
    s = prob.s[64:65]
    x = torch.from_numpy(W.random_complex_vectors(1, 3 * ne) * 1e-6).cuda()
    y = torch.zeros_like(x)
    for _ in range(2):
        P.bem_apply(c.h, s, x, y, P.BEM_PREC_FP32, P.BEM_APPLY_A)
    torch.cuda.synchronize()
    print("single-frequency kernel case done: units", ne * (ne - 1) * 4)


def kernel_case():
    """Small case for ncu captures of the operator kernels: the 5120-triangle cavity, 24
    consecutive benchmark frequencies (s_52 .. s_75, equally spaced: the FP32 operator runs them
    through its recurrence kernel as two CTA groups of 12), one FP32 operator application and
    one float-float refinement residual, each after a warm-up call."""
    import torch

    import paper_1511_04355_gb300 as P

    prob = W.spherical_cavity(level=LEVEL, n_freq=N_FREQ, T=T_WIN, sigma=SIGMA)
    c = P.Context(0)
    c.set_mesh(prob.verts, prob.tris)
    m = prob.material
    c.set_material(m.mu, m.nu, m.rho)
    c.set_bc(prob.bc_type, prob.bc_value)
    ne = len(prob.tris)
    s = prob.s[52:76]
    x = torch.from_numpy(W.random_complex_vectors(len(s), 3 * ne) * 1e-6).cuda()
    y = torch.zeros_like(x)
    for _ in range(2):
        P.bem_apply(c.h, s, x, y, P.BEM_PREC_FP32, P.BEM_APPLY_A)
        P.bem_residual(c.h, s, x, y, P.BEM_RESID_DF64)
        P.bem_apply(c.h, s, x, y, P.BEM_PREC_FP64, P.BEM_APPLY_A)
    torch.cuda.synchronize()
    print("kernel case done: units per far launch", len(s) * ne * (ne - 1) * 4)


def profile_step():
    """One mixed solve of the benchmark step (128 frequencies, tol 1e-6) with the library's
    per-class kernel timing on: prints the far32 launches and their frequency-launches, i.e. the
    units (x ne (ne - 1) 4) an ncu capture of this command's far32 launches divides by."""
    import torch

    import paper_1511_04355_gb300 as P

    prob = W.spherical_cavity(level=LEVEL, n_freq=N_FREQ, T=T_WIN, sigma=SIGMA)
    c = P.Context(0)
    c.set_mesh(prob.verts, prob.tris)
    m = prob.material
    c.set_material(m.mu, m.nu, m.rho)
    c.set_bc(prob.bc_type, prob.bc_value, P.BEM_PROFILE_STEP)
    c.set_options(precision=P.BEM_PREC_MIXED, tol=TOL)
    ne = len(prob.tris)
    c.profile(True)
    x, info = c.solve(prob.s)
    kt = c.kernel_times()
    torch.cuda.synchronize()
    n32, ms32, fl32 = kt["far32"]
    print(json.dumps({"far32_launches": n32, "far32_freq_launches": fl32,
                      "far32_units": fl32 * ne * (ne - 1) * 4, "far32_ms": ms32,
                      "kernel_ms": {k: v[1] for k, v in kt.items()},
                      "gmres_iterations": int(info["iterations"].sum())}))


def workload_uneven():
    """The uneven-instance workload: 16 ellipsoidal cavities (icosphere levels 2-5, 320-20480
    triangles, their own materials), 64 frequencies each, all solved together through
    bem_solve_batch (one host worker and one stream per context), once with the fixed FP32
    launch shape and once with the shapes of the committed tuning table (far32_tuning.txt)."""
    import torch

    import paper_1511_04355_gb300 as P

    insts = W.uneven_instances(n_inst=16, levels=(2, 3, 4, 5))
    s = W.fsm_frequencies(T_WIN, SIGMA, 64)
    ctxs = []
    for v, f, mat in insts:
        c = P.Context(0, tuning=False)
        c.set_mesh(v, f)
        c.set_material(mat.mu, mat.nu, mat.rho)
        c.set_bc(np.zeros(len(f), np.int8), W.pressure_pattern(v, f), P.BEM_PROFILE_STEP)
        c.set_options(precision=P.BEM_PREC_MIXED, tol=TOL)
        ctxs.append(c)
    outs = [np.zeros((len(s), 3 * c.ne), np.complex128) for c in ctxs]
    # warm-up (allocations, module load)
    P.bem_solve_batch([(c.h, s[:2], o[:2]) for c, o in zip(ctxs, outs)])
    torch.cuda.synchronize()
    n = len(s) * len(ctxs)
    runs = {}
    for mode in ("fixed", "tuned"):
        for c in ctxs:
            if mode == "fixed":
                P.bem_set_tuning(c.h, [])
            else:
                P.bem_load_tuning(c.h, P.TUNING_TABLE)
        t0 = time.perf_counter()
        res = P.bem_solve_batch([(c.h, s, o) for c, o in zip(ctxs, outs)])
        t_bat = time.perf_counter() - t0
        ok = all((info["status"] == 0).all() and (info["residual"] <= TOL).all() for _, info in res)
        runs[mode] = {"seconds": t_bat, "solves_per_s": n / t_bat, "all_certified": bool(ok),
                      "iterations_total": int(sum(int(i["iterations"].sum()) for _, i in res))}
        print(json.dumps({"mode": mode, **runs[mode]}), file=sys.stderr, flush=True)
    line = {"workload": "16 uneven ellipsoidal cavities (icosphere levels 2-5, 320-20480 triangles), "
                        "64 frequencies each, mixed path to 1e-6, solved together by bem_solve_batch",
            "triangles": [len(f) for _, f, _ in insts], "solves": n,
            "fixed_launch_shape": runs["fixed"], "autotuned_launch_shapes": runs["tuned"],
            "speedup_tuned_vs_fixed": runs["fixed"]["seconds"] / runs["tuned"]["seconds"]}
    print(json.dumps(line), flush=True)


AFS_TOL = TOL    # residual tolerance of the AFS samples (--afs-tol; see afs_vs_fsm)
AFS_WARM = None  # warm start of the AFS samples (--afs-warm; None: the workload's own choice)


HMATRIX = None   # bem_hmatrix_params fields for the AFS-vs-FSM workloads (--hmatrix)


def afs_vs_fsm(label, pb, dofs, n_orf, period, nc, J0, warm, restart=200, extra=None, max_samples=None):
    """AFS (Sec. 3) against the FSM (Sec. 2.2) on one problem through the library: the FSM solves
    the nc frequencies eta + i k 2 pi / period at once; AFS samples the same band [0, Omega],
    Omega = (nc - 1) 2 pi / period, adaptively, with its first n_orf unknowns as observation
    responses and the rest as test unknowns.  eta = 3 ln(10) / period (Sec. 2.2 with the kappa =
    3 of Sec. 4).  The transients are compared over the first half of the period, against the
    FSM with the Hanning window (the paper's) and without it (the same band-limited information
    as the fit: the window smooths what the truncated band leaves).  The FSM's solves stop at
    the benchmark tolerance, AFS's at AFS_TOL (the same by default; 1e-8 was measured too: on
    the low bands AFS then took 47 against 40 samples on the porous block and the same 34 on
    the Example-3 block, and on the full bands it did not converge either way).  Prints one
    JSON line."""
    import paper_1511_04355_gb300 as P

    v, f, m = pb["verts"], pb["tris"], pb["material"]
    c = P.Context(0)
    c.set_mesh(v, f)
    c.set_material(m.mu, m.nu, m.rho)
    c.set_bc(pb["bc_type"], pb["bc_value"], P.BEM_PROFILE_STEP)
    c.set_options(precision=P.BEM_PREC_MIXED, tol=TOL, restart=restart, max_iters=6000, max_refine=20,
                  warm_start=P.BEM_WARM_ZERO)
    if HMATRIX is not None:
        c.set_hmatrix(True, **HMATRIX)
        label += "; H-matrix far field in the FP32 inner operator"
    eta = 3.0 * math.log(10.0) / period
    omega = (nc - 1) * 2.0 * math.pi / period
    t = np.linspace(0.0, 0.5 * period, 201)
    # the FSM: one batched solve of the nc frequencies, inverted with and without the window
    t0 = time.perf_counter()
    x, finfo = c.solve(eta + 1j * np.arange(nc) * 2.0 * math.pi / period)
    h = np.ascontiguousarray(x[:, dofs])
    fsm_w = c.fsm_eval(h, eta, period, t, 1)
    t_fsm = time.perf_counter() - t0
    fsm_n = c.fsm_eval(h, eta, period, t, 0)
    del x
    print(json.dumps({"label": label, "fsm_seconds": t_fsm, "triangles": len(f),
                      "fsm_iterations": int(finfo["iterations"].sum())}), file=sys.stderr, flush=True)
    if AFS_WARM is not None:
        warm = AFS_WARM
    c.set_options(precision=P.BEM_PREC_MIXED, tol=AFS_TOL, restart=restart, max_iters=6000, max_refine=20,
                  warm_start=warm)
    prm = P.bem_default_afs_params(eta=eta, omega_max=omega, T=period, J0=J0, max_samples=max_samples or nc)
    t0 = time.perf_counter()
    afs_out, info = c.afs(prm, dofs[:n_orf], dofs[n_orf:], t)
    t_afs = time.perf_counter() - t0

    def rel(a, b):
        return (np.sqrt(np.sum((a - b) ** 2, axis=0) / np.sum(b ** 2, axis=0))).tolist()

    line = {"workload": label, "triangles": len(f), "unknowns": 3 * len(f),
            "eta": eta, "period": period, "omega_max": omega,
            "fsm": {"n_c": nc, "seconds": t_fsm, "gmres_iterations": int(finfo["iterations"].sum())},
            "fsm_tol": TOL, "afs_tol": AFS_TOL,
            "afs": {"n_c": int(info["n_samples"]), "seconds": t_afs, "poles": len(info["poles"]),
                    "converged": bool(int(info["n_samples"]) < (max_samples or nc)),
                    "E1": float(info["E1"][-1]), "E2": float(info["E2"][-1]),
                    "seconds_solve": info["seconds_solve"], "seconds_fit": info["seconds_fit"],
                    "seconds_train": info["seconds_train"],
                    "gmres_iterations": int(np.sum(info["gmres_iters"])),
                    "warm_start": {0: "zero", 1: "nearest", 2: "mlp", 3: "vf"}[warm]},
            "afs_vs_fsm_rel_l2": {"hanning": rel(afs_out, fsm_w), "no_window": rel(afs_out, fsm_n)},
            "fsm_hanning_vs_no_window_rel_l2": rel(fsm_w, fsm_n),
            "nc_ratio_fsm_over_afs": nc / max(int(info["n_samples"]), 1)}
    if extra:
        line.update(extra)
    if HMATRIX is not None:
        line["hmatrix"] = {"params": HMATRIX, "info": c.hmatrix_info()}
    print(json.dumps(line), flush=True)
    c.close()


def workload_porous_afs(full=False, lowband=False):
    """The porous-block workload: a 1 m block with 27 seeded spherical voids (radii 0.08-0.15 m),
    traction on z = 0, z = 1 fixed; the step response of six unknowns by a 256-frequency FSM and
    by AFS over the same band.  full: the ~30000-triangle recipe (42 x 42 grid per face, level-2
    voids), 256 frequencies over a 40 ms period (Omega ~ 40000 rad/s); else a reduced mesh (20 x
    20 per face, level-1 voids, 6960 triangles), 128 frequencies over a 50 ms period (Omega =
    127 x 2 pi / 0.05 ~ 16000 rad/s, ~5.5 elements per shear wavelength); lowband: the mesh
    chosen by full, 64 frequencies over a 0.1 s period (Omega ~ 4000 rad/s, a band holding a few
    elastic modes of the block).  GMRES(200): box problems with a fixed face need hundreds of
    iterations at the upper frequencies, where GMRES(50) restarts stall."""
    if full:
        pb = W.porous_block(n=(42, 42, 42), n_voids=27, void_level=2)
    else:
        pb = W.porous_block(n=(20, 20, 20), n_voids=27, void_level=1)
    v, f = pb["verts"], pb["tris"]
    face = pb["face"]
    cent = v[f].mean(axis=1)

    def nearest(mask, target):
        idx = np.flatnonzero(mask)
        return int(idx[np.argmin(np.linalg.norm(cent[idx] - target, axis=1))])
    voids = np.flatnonzero(face < 0)
    dofs = np.array([3 * nearest(face == 4, [0.5, 0.5, 0.0]) + 2,       # loaded face, u_z
                     3 * nearest(face == 0, [0.0, 0.5, 0.5]) + 0,       # side face, u_x
                     3 * int(voids[0]) + 2, 3 * int(voids[len(voids) // 2]) + 2,
                     3 * nearest(face == 4, [0.25, 0.75, 0.0]) + 2,
                     3 * int(voids[-1]) + 2])
    period, nc = (2 * T_WIN, 256) if full else (0.05, 128)
    if lowband:   # the same mesh over a band holding few modes: 64 frequencies over a 0.1 s period
        period, nc = 0.1, 64
    label = (f"porous block 1x1x1 m, 27 voids, {len(f)} triangles ({3 * len(f)} unknowns), step traction "
             "on z=0, z=1 fixed")
    afs_vs_fsm(label, pb, dofs, 4, period, nc, 8, 1, max_samples=nc + nc // 2)


def workload_example3(warm=0, n=(12, 12, 18), void_level=1, nc=240):
    """The paper's third example (Sec. 4, Example 3): the 1 x 1 x 1.5 m aluminium block with 98
    cavities of radius 0.072 m, fixed on z = 1.5, step traction on z = 0; period T = 0.035 s, FSM
    with N_s = 478 (N_c = 240) against AFS with the paper's parameters (J0 = 16, alpha 2.0 / 2.3,
    E1 < 1e-4, E2 < 2e-3, J_c = 3) and six observation responses (two tractions on the fixed
    face, four displacements), two test unknowns (u_z on the loaded face, t_z on the fixed face).
    The paper reports N_c = 240 (FSM) against 61 (AFS) for its 18080 quadratic elements.  nc: FSM
    frequencies N_s / 2 + 1 over the same period (57: a band of ~10000 rad/s, a few modes)."""
    pb = W.example3_block(n=n, void_level=void_level)
    v, f = pb["verts"], pb["tris"]
    face = pb["face"]
    cent = v[f].mean(axis=1)

    def nearest(mask, target):
        idx = np.flatnonzero(mask)
        return int(idx[np.argmin(np.linalg.norm(cent[idx] - target, axis=1))])
    cav = np.flatnonzero(face < 0)
    dofs = np.array([3 * nearest(face == 5, [0.3, 0.4, 1.5]) + 2,        # t_z, fixed face
                     3 * nearest(face == 5, [0.7, 0.2, 1.5]) + 2,        # t_z, fixed face
                     3 * nearest(face == 4, [0.5, 0.5, 0.0]) + 2,        # u_z, loaded face
                     3 * nearest(face == 0, [0.0, 0.5, 0.75]) + 0,       # u_x, side face
                     3 * int(cav[len(cav) // 3]) + 2,                    # u_z, a cavity wall
                     3 * nearest(face == 2, [0.5, 0.0, 1.0]) + 1,        # u_y, side face
                     3 * nearest(face == 4, [0.74, 0.34, 0.0]) + 2,      # test: u_z, loaded face
                     3 * nearest(face == 5, [0.6, 0.8, 1.5]) + 2])       # test: t_z, fixed face
    label = (f"block 1x1x1.5 m with 98 cavities r=0.072 m (Example 3), aluminium, {len(f)} triangles "
             f"({3 * len(f)} unknowns), fixed z=1.5, step traction on z=0")
    afs_vs_fsm(label, pb, dofs, 6, 0.035, nc, 16, warm, extra={"paper_nc": {"fsm": 240, "afs": 61}},
               max_samples=nc + nc // 3)


def hm_kernel_case():
    """The H-matrix apply at capture size: a 2 x 1 x 1 m porous block, 32 x 16 x 16 face grids and
    10 voids (level-1 icospheres, 5920 triangles; about 1 GB of factors, several times the L2),
    the FP32 operator applied at one frequency (k = 7 of the large workload's list) with the
    H-matrix far field, twice (the first call builds the factors).  Prints the partition and
    factor sizes."""
    import paper_1511_04355_gb300 as P

    pb = W.porous_block(L=(2.0, 1.0, 1.0), n=(32, 16, 16), n_voids=10, radii=(0.08, 0.1), void_level=1)
    period = 2 * T_WIN
    s = np.array([3.0 * math.log(10.0) / period + 1j * 7 * 2.0 * math.pi / period])
    c = P.Context(0)
    c.set_mesh(pb["verts"], pb["tris"])
    m = pb["material"]
    c.set_material(m.mu, m.nu, m.rho)
    c.set_bc(pb["bc_type"], pb["bc_value"], P.BEM_PROFILE_STEP)
    c.set_hmatrix(True, leaf=32, eta=2.0, max_block=512, max_rank=128, eps=1e-4)
    rng = np.random.default_rng(W.SEED)
    x = rng.standard_normal((1, 3 * len(pb["tris"]))) + 1j * rng.standard_normal((1, 3 * len(pb["tris"])))
    c.apply(s, x, precision=P.BEM_PREC_FP32)
    c.profile(True)
    c.apply(s, x, precision=P.BEM_PREC_FP32)
    kt = c.kernel_times()
    print(json.dumps({"triangles": len(pb["tris"]), "info": c.hmatrix_info(), "happly_ms": kt["happly"][1]}))


def workload_large(n_freq=8, hmatrix=None):
    """The large porous solid: a 2 x 1 x 1 m block with 200 seeded spherical voids (radii 0.05-0.1
    m, level-2 icospheres) and 84 x 42 x 42 face grids, 99280 triangles (297840 complex unknowns);
    step traction 1e6 Pa on z = 0, z = 1 fixed.  One batched mixed-precision solve (tol 1e-6,
    GMRES(100)) of the first n_freq frequencies s_k = eta + i k 2 pi / P with P = 40 ms and eta =
    3 ln(10) / P (Sec. 2.2, kappa = 3) through bem_solve_frequencies.  Prints one JSON line with
    solves/s, GMRES iterations, refinements and the device memory the solve held.  hmatrix: a dict
    of bem_hmatrix_params fields; the FP32 inner operator then uses the H-matrix far field (the
    FP64-class residual stays the exact operator)."""
    import torch

    import paper_1511_04355_gb300 as P

    pb = W.porous_block(L=(2.0, 1.0, 1.0), n=(84, 42, 42), n_voids=200, radii=(0.05, 0.1), void_level=2)
    v, f, m = pb["verts"], pb["tris"], pb["material"]
    period = 2 * T_WIN
    eta = 3.0 * math.log(10.0) / period
    s = eta + 1j * np.arange(n_freq) * 2.0 * math.pi / period
    c = P.Context(0)
    t0 = time.perf_counter()
    c.set_mesh(v, f)
    c.set_material(m.mu, m.nu, m.rho)
    c.set_bc(pb["bc_type"], pb["bc_value"], P.BEM_PROFILE_STEP)
    t_setup = time.perf_counter() - t0
    c.set_options(precision=P.BEM_PREC_MIXED, tol=TOL, restart=100, max_iters=3000, max_refine=12)
    if hmatrix is not None:
        c.set_hmatrix(True, **hmatrix)
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    free0, total = torch.cuda.mem_get_info()
    x = torch.zeros((n_freq, 3 * len(f)), dtype=torch.complex128, device="cuda")
    c.profile(True)
    t0 = time.perf_counter()
    _, info = P.bem_solve_frequencies(c.h, torch.from_numpy(s).cuda(), x, allow_not_converged=True)
    torch.cuda.synchronize()
    t_solve = time.perf_counter() - t0
    kt = c.kernel_times()
    free1, _ = torch.cuda.mem_get_info()
    ne = len(f)
    n32, ms32, fl32 = kt["far32"]
    line = {"workload": f"porous block 2x1x1 m, 200 voids, {ne} triangles ({3 * ne} complex unknowns), step "
                        f"traction on z=0, z=1 fixed; {n_freq} frequencies eta + i k 2 pi / {period}",
            "triangles": ne, "unknowns": 3 * ne, "frequencies": n_freq, "eta": eta,
            "seconds_setup": t_setup, "seconds_solve": t_solve, "solves_per_s": n_freq / t_solve,
            "status": info["status"].tolist(), "residual": info["residual"].tolist(),
            "gmres_iterations": info["iterations"].tolist(), "refinements": info["refinements"].tolist(),
            "device_bytes_in_use_after_solve": int(total - free1),
            "far32": {"launches": n32, "ms": ms32,
                      "tflops_executed": fl32 * ne * (ne - 1) * 4 * FLOPS_EXEC_PER_UNIT_FAR32 / (ms32 / 1e3) / 1e12
                      if ms32 > 0 else None},
            "kernel_ms": {k: v[1] for k, v in kt.items()}}
    if hmatrix is not None:
        hi = c.hmatrix_info()
        line["workload"] += "; H-matrix far field in the FP32 inner operator"
        line["hmatrix"] = {"params": hmatrix, "info": hi,
                           "apply": {"launches": kt["happly"][0], "ms": kt["happly"][1],
                                     "frequency_applies": kt["happly"][2]},
                           "build_ms": kt["hbuild"][1]}
        na = kt["happly"][2]
        if na > 0 and hi["frequencies"] > 0:
            # the low-rank factors of one frequency, read once per frequency application
            line["hmatrix"]["factor_bytes_per_frequency"] = hi["factor_bytes"] / hi["frequencies"]
            line["hmatrix"]["ms_per_frequency_apply"] = kt["happly"][1] / na
    print(json.dumps(line), flush=True)


def main():
    global AFS_TOL, AFS_WARM, HMATRIX
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--kernel-case", action="store_true",
                    help="run only the small operator/residual case used for ncu captures")
    ap.add_argument("--afs-warm", choices=["zero", "nearest", "mlp", "vf"], default=None,
                    help="warm start of the AFS solves in the AFS-vs-FSM workloads (default nearest)")
    ap.add_argument("--afs-tol", type=float, default=AFS_TOL,
                    help="residual tolerance of the AFS samples in the AFS-vs-FSM workloads")
    ap.add_argument("--hm-eps", type=float, default=1e-4,
                    help="cross-approximation tolerance of the H-matrix workloads")
    ap.add_argument("--hm-max-freqs", type=int, default=2,
                    help="frequencies whose H-matrix factors are held at once (H-matrix workloads)")
    ap.add_argument("--hmatrix", action="store_true",
                    help="AFS-vs-FSM workloads: the FP32 inner operator uses the H-matrix far field")
    ap.add_argument("--hm-kernel-case", action="store_true",
                    help="run only the H-matrix apply case used for ncu captures")
    ap.add_argument("--kernel-case-single", action="store_true",
                    help="run only the single-frequency FP32 operator case used for ncu captures")
    ap.add_argument("--profile-step", action="store_true",
                    help="run one benchmark solve with kernel counts (for ncu instruction counters)")
    ap.add_argument("--workload", choices=["uneven", "porous-afs", "porous-afs-full", "example3",
                                           "example3-mlp", "large", "large-hmatrix", "porous-afs-lowband",
                                           "porous-afs-full-lowband", "example3-lowband"],
                    help="run one of the other workloads instead of the benchmark (own JSON line)")
    args = ap.parse_args()
    AFS_TOL = args.afs_tol
    if args.hmatrix:
        HMATRIX = dict(leaf=32, eta=2.0, max_block=512, max_rank=128, eps=args.hm_eps, max_freqs=args.hm_max_freqs)
    if args.afs_warm:
        AFS_WARM = {"zero": 0, "nearest": 1, "mlp": 2, "vf": 3}[args.afs_warm]
    if args.kernel_case:
        kernel_case()
        return
    if args.kernel_case_single:
        kernel_case_single()
        return
    if args.profile_step:
        profile_step()
        return
    if args.workload == "uneven":
        workload_uneven()
        return
    if args.workload in ("porous-afs", "porous-afs-full", "porous-afs-lowband", "porous-afs-full-lowband"):
        workload_porous_afs(full=args.workload in ("porous-afs-full", "porous-afs-full-lowband"),
                            lowband=args.workload.endswith("lowband"))
        return
    if args.workload == "example3-lowband":
        workload_example3(warm=1, nc=57)   # N_s = 112 over T = 0.035 s: Omega ~ 10000 rad/s
        return
    if args.hm_kernel_case:
        hm_kernel_case()
        return
    if args.workload == "large":
        workload_large()
        return
    if args.workload == "large-hmatrix":
        workload_large(hmatrix=dict(leaf=32, eta=2.0, max_block=512, max_rank=128, eps=args.hm_eps,
                                    max_freqs=args.hm_max_freqs))
        return
    if args.workload in ("example3", "example3-mlp"):
        workload_example3(warm=2 if args.workload == "example3-mlp" else 1)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
