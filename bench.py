"""Benchmark of the pipe-flow time step on GB300 (one JSON line on stdout).

Workload: the medium single-run configuration -- N=48 radial points, |k|<32,
m<24, m_p=2, Re=2400, alpha=1.25, dt=0.005, seeded puff-like perturbation of
amplitude 0.1 -- one "step" = one full predictor-corrector time step
(2 nonlinear evaluations + 2 banded-solve passes) of that grid.  The state
fits in L2, so L2 is flushed between timed steps (a 256 MB write, then a
256 MB read of another buffer, so the lines left in L2 are clean and no
write-back of the flush lands inside the step) and each step is timed alone
with CUDA events on the launching stream.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision 0|1] [--impl reference]

N > 1 (torchrun, one rank per GPU): independent replicas, no collective on
the data path; time = max over ranks; value = all ranks' steps / that time.
--impl reference times the CPU oracle (the plain FP64 restatement of the
method) on the host cores for the same workload and metric.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "timesteps/s & GDOF-steps/s per grid, mixed vs FP64 on 1 GB300; % HBM roofline"
WORKLOAD = "medium"
L2_FLUSH_BYTES = 256 << 20


def workload_params():
    from paper_1705_03838_gb300 import inputs

    w = inputs.WORKLOADS[WORKLOAD]
    return w


def dof(w):
    return 3 * w["N"] * (2 * w["K"] - 1) * (2 * w["M"] - 1)


def config_dict(w, precision):
    return {
        "workload": (f"pipe medium: N={w['N']} |k|<{w['K']} m<{w['M']} m_p={w['m_p']} "
                     f"Re={w['Re']:g} alpha={w['alpha']} dt={w['dt']} amp={w['amplitude']}"),
        "grid": f"{3 * w['K']}x{3 * w['M']} (z x theta) per radial point",
        "dof": dof(w),
        "precision": "fp64" if precision == 0 else "mixed (fp32 transforms, fp64 solves)",
        "l2": "flushed before every timed step (256 MB write, then 256 MB read of a second buffer)",
        "parallelism": "replicas (one trajectory per GPU)",
    }


# ------------------------------------------------------------------ algorithmic costs
def kernel_costs(w, precision=1):
    """Algorithmic flops and bytes per launch, per kernel.

    FFT flops use 2.5 n log2 n per real 2-D transform of n = 9KM points,
    split between z (log2 3K) and theta (log2 3M) parts.  The solve counts,
    per mode and radial row: div N_eff (48), d_r p (36), right-hand sides (30),
    final update and influence correction (36), and 8 real banded
    substitutions (2 nl + 2 nu + 1 each, nl/nu the row's band widths).  In FP64
    steps the solve launches also take the curl of their output (A1) for the
    next nonlinear evaluation, so their cost includes the curl's."""
    N, K, M = w["N"], w["K"], w["M"]
    nz, nth, nk = 3 * K, 3 * M, 2 * K - 1
    n = nz * nth
    F = N * nk * M  # complex per spectral field
    P = N * nz * M  # complex per half-physical field
    lz, lt = math.log2(nz), math.log2(nth)
    lo = [min(max(i - 4, 0), N - 9) for i in range(N)]
    band = sum(2 * (i - lo[i]) + 2 * (min(i + 4, N - 1) - i) + 1 for i in range(N))
    modes = nk * M
    solve = modes * (N * (48 + 36 + 30 + 36) + 8 * band)
    return {
        "curl": {"flops": F * (2 * 9 * 4 + 30), "bytes": 16 * (3 * F + 6 * F)},
        "zsynth": {"flops": 6 * N * 2.5 * n * lz, "bytes": 16 * (6 * F + 6 * P)},
        "product": {"flops": 9 * N * 2.5 * n * lt + 9 * N * n, "bytes": 16 * (6 * P + 3 * P)},
        "zanalysis": {"flops": 3 * N * 2.5 * n * lz, "bytes": 16 * (3 * P + 3 * F)},
        "solve": {"flops": solve + (F * (2 * 9 * 4 + 30) if precision == 0 else 0),
                  "bytes": 16 * (3 * F * 3 + 3 * F + (6 * F if precision == 0 else 0))},
    }


# dram__bytes_read.sum + dram__bytes_write.sum per launch of the current
# kernels on the medium workload (one ncu capture each, summarised in the
# named profile), keyed by (kernel, precision of the step)
PROFILED_DRAM_BYTES = {("solve", 1): 20.78e6}  # kernels changed since a capture are left out
PROFILE_FILES = {"solve": "profiles/k_solve_medium.md", "product": "profiles/transforms_medium.md"}


# which arithmetic bounds each kernel: FP64 for the solve and the curl (both
# precisions), the transforms follow the precision
def kernel_peak(name, precision):
    if precision == 1 and name in ("zsynth", "product", "zanalysis"):
        return FP32_PEAK_TFLOPS, "FP32 from unit counts (152 SMs x 128 lanes x 2 flops x 2.07 GHz)"
    return FP64_PEAK_TFLOPS, "FP64 from unit counts (152 SMs x 2 DFMA/clk x 2 flops x 2.07 GHz)"


def step_algorithmic_bytes(w, precision):
    """Minimum HBM bytes per step: spectral fields only (528 F FP64, 432 F mixed)."""
    F = w["N"] * (2 * w["K"] - 1) * w["M"]
    return (528 if precision == 0 else 432) * F


def max_over_ranks(x, dist=None, device="cpu"):
    """The largest per-rank value over the ranks of the process group (x
    itself without one): the job's time is its slowest rank's."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, seconds):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (each rank processes the same number of units)."""
    return units_per_rank * world / seconds


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# Peaks from unit counts at the 2.07 GHz maximum SM clock: FP64 152 SMs x 2
# DFMA/clk x 2 flops (FMA probe on this GPU: 1.20 TFLOP/s); FP32 152 SMs x 128
# lanes x 2 flops (probe: 70 TFLOP/s).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.path = None
        self.gpu = gpu_index

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.close()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = max(smax, float(parts[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle timing
def oracle_timing(seconds_budget=20.0, max_steps=None):
    """Time the CPU oracle (single thread) on the same workload in a fresh
    process; returns (steps/s, steps timed, setup seconds)."""
    budget = seconds_budget
    code = f"""
import os, sys, time, json
sys.path.insert(0, {ROOT!r})
from oracle.opf_oracle import Oracle, Params
from paper_1705_03838_gb300 import inputs
w = inputs.WORKLOADS[{WORKLOAD!r}]
o = Oracle(Params(w['N'], w['K'], w['M'], w['m_p'], w['alpha'], w['Re'], w['dt']))
U = inputs.workload_state({WORKLOAD!r})
t0 = time.time(); U = o.step(U, 1); setup = time.time() - t0
n = 0; t0 = time.time()
while True:
    U = o.step(U, 1); n += 1
    el = time.time() - t0
    if el > {budget} or ({max_steps!r} is not None and n >= {max_steps!r}):
        break
print(json.dumps({{"steps": n, "seconds": el, "setup": setup}}))
"""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError("oracle timing failed: " + r.stderr[-2000:])
    res = json.loads(r.stdout.strip().splitlines()[-1])
    return res["steps"] / res["seconds"], res["steps"], res["setup"], res["seconds"]


def oracle_timing_all_cores(seconds_budget=10.0):
    """The oracle on all host cores: one single-threaded oracle process per
    core (memory permitting), each stepping its own seeded trajectory of the
    same workload; returns (aggregate steps/s, processes, total steps)."""
    nproc = os.cpu_count() or 1
    try:  # ~1.2 GB per medium oracle process (LU factors of 1512 modes)
        avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
        nproc = max(1, min(nproc, int(avail // (1.5 * 2 ** 30))))
    except (ValueError, OSError, AttributeError):
        pass
    code = f"""
import sys, time, json
sys.path.insert(0, {ROOT!r})
from oracle.opf_oracle import Oracle, Params
from paper_1705_03838_gb300 import inputs
w = inputs.WORKLOADS[{WORKLOAD!r}]
rank = int(sys.argv[1])
o = Oracle(Params(w['N'], w['K'], w['M'], w['m_p'], w['alpha'], w['Re'], w['dt']))
U = inputs.seeded_state(w['N'], w['K'], w['M'], w['m_p'], w['alpha'], w['amplitude'], w['seed'] + rank,
                        w['envelope'])
U = o.step(U, 1)
n = 0; t0 = time.time()
while True:
    U = o.step(U, 1); n += 1
    el = time.time() - t0
    if el > {seconds_budget}:
        break
print(json.dumps({{"steps": n, "seconds": el}}))
"""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    procs = [subprocess.Popen([sys.executable, "-c", code, str(i)], stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True, env=env) for i in range(nproc)]
    rate, steps = 0.0, 0
    for p in procs:
        out, err = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("oracle timing failed: " + err[-2000:])
        res = json.loads(out.strip().splitlines()[-1])
        rate += res["steps"] / res["seconds"]
        steps += res["steps"]
    return rate, nproc, steps


def oracle_small_full():
    """The small workload in full (100 steps, N=32, |k|<16, m<16) on one core."""
    code = f"""
import sys, time, json
sys.path.insert(0, {ROOT!r})
from oracle.opf_oracle import Oracle, Params
from paper_1705_03838_gb300 import inputs
w = inputs.WORKLOADS['small']
o = Oracle(Params(w['N'], w['K'], w['M'], w['m_p'], w['alpha'], w['Re'], w['dt']))
U = inputs.workload_state('small')
t0 = time.time(); U = o.step(U, 100); el = time.time() - t0
print(json.dumps({{"steps": 100, "seconds": el, "energy": [float(x) for x in o.energy(U)]}}))
"""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError("oracle timing failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


LARGE_ORACLE_NOTE = ("large workload (N=128, |k|<128, m<128) not stepped on the host: the oracle's dense "
                     "solve factors 32,640 complex systems of order 513 per dt (~47 TFLOP of LU), hours "
                     "per step; it is checked instead on its nonlinear term and sampled-mode solves")


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    per_step = None
    # bounded sample: as many full oracle steps as fit in ~2 minutes, at most K
    sps, n, setup, secs = oracle_timing(seconds_budget=min(120.0, 1.0 + 0.7 * args.steps),
                                        max_steps=args.steps)
    gd = dof(w)
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": sps,
        "unit": "timesteps/s",
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1000.0 / sps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": config_dict(w, 0),
        "gdof_steps_per_s": sps * gd / 1e9,
        "cpu_baseline": {"value": sps, "unit": "timesteps/s", "cores": 1, "kind": "oracle",
                         "sample": f"{n} full oracle steps of the medium workload after 1 setup step "
                                   f"({setup:.1f} s, LU factorisation), {secs:.1f} s"},
        "e2e": {"value": sps, "unit": "timesteps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
ENSEMBLE_SHAPES = [(32, 16, 16)] * 96 + [(48, 24, 24)] * 96 + [(64, 32, 32)] * 64


def ensemble_shapes(count):
    """The ensemble's resolutions in its 96 : 96 : 64 proportion, count in all
    (256 = the full workload; smaller counts for profiling)."""
    if count >= len(ENSEMBLE_SHAPES):
        return ENSEMBLE_SHAPES
    a = max(1, round(count * 96 / 256))
    c = max(1, round(count * 64 / 256))
    b = max(1, count - a - c)
    return [(32, 16, 16)] * a + [(48, 24, 24)] * b + [(64, 32, 32)] * c


def run_ensemble(args):
    """Batched-ensemble workload: 256 trajectories of uneven resolution
    (96 x N=32 |k|<16 m<16, 96 x N=48 |k|<24 m<24, 64 x N=64 |k|<32 m<32),
    Re uniform in [1800, 2600], perturbation amplitude log-uniform in
    [1e-3, 1e-1], mixed precision, all stepped in one CUDA graph per step.
    The working set (~10 GB) exceeds L2, so no flush is needed."""
    import torch

    from paper_1705_03838_gb300 import build as _build, inputs, opf

    torch.cuda.set_device(0)
    _build.build()
    shapes = ensemble_shapes(args.ens_count)
    n = len(shapes)
    seed = 1705038383
    U = inputs.uniforms(seed, 2 * n)
    Re = [1800.0 + 800.0 * U[2 * i] for i in range(n)]
    amp = [10.0 ** (-3.0 + 2.0 * U[2 * i + 1]) for i in range(n)]
    Ns, Ks, Ms = zip(*shapes)
    alpha, dt = 1.25, 0.005
    t0 = time.time()
    e = opf.opf_ens_create(Ns, Ks, Ms, [1] * n, [alpha] * n, Re, [dt] * n)
    setup_s = time.time() - t0
    stream = torch.cuda.current_stream()
    opf.opf_ens_set_stream(e, stream.cuda_stream)
    opf.opf_ens_set_option(e, "precision", args.precision)
    t0 = time.time()
    for i, (N, K, M) in enumerate(shapes):
        opf.opf_ens_set_state(e, i, inputs.seeded_state(N, K, M, 1, alpha, amp[i], seed + i))
    inputs_s = time.time() - t0
    if args.autotune:
        opf.opf_ens_set_option(e, "autotune", 1)
    opf.opf_ens_step(e, args.warmup)
    # kernel shares from untimed instrumented steps; the timed steps carry
    # event records around the solve only
    opf.opf_ens_set_option(e, "timing", 1)
    opf.opf_ens_kernel_times(e, reset=True)
    opf.opf_ens_step(e, 2)
    kt_all = opf.opf_ens_kernel_times(e, reset=True)
    opf.opf_ens_set_option(e, "timing", 2)
    opf.opf_ens_set_option(e, "timed_kernel", 4)
    opf.opf_ens_step(e, 1)
    opf.opf_ens_kernel_times(e, reset=True)
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    opf.opf_ens_step(e, args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = ev0.elapsed_time(ev1)
    kt_live = opf.opf_ens_kernel_times(e, reset=True)
    kt = {k: (v[0] / max(1, v[1]), 1) for k, v in kt_all.items()}  # per-launch averages
    kt["solve"] = (kt_live["solve"][0] / max(1, kt_live["solve"][1]), 1)
    firsts = [shapes.index(sh) for sh in dict.fromkeys(shapes)]
    E = [opf.opf_ens_energy(e, i) for i in firsts]
    steps_per_s = args.steps / (total_ms / 1000.0)
    dofs = sum(3 * N * (2 * K - 1) * (2 * M - 1) for N, K, M in shapes)
    Fsum = sum(N * (2 * K - 1) * M for N, K, M in shapes)
    peaks, peak_kind = load_peaks()
    algo_bytes = (528 if args.precision == 0 else 432) * Fsum
    flops = {}
    for (N, K, M), cnt in ((sh, shapes.count(sh)) for sh in dict.fromkeys(shapes)):
        c = kernel_costs({"N": N, "K": K, "M": M})
        for k, v in c.items():
            flops[k] = flops.get(k, 0.0) + cnt * v["flops"]
    dom = max(kt, key=lambda k: kt[k][0])
    dom_ms = kt[dom][0] / max(1, kt[dom][1]) * len(set(shapes))  # one launch per shape group per slot
    pk, src = kernel_peak(dom, args.precision)
    ach = flops[dom] / (dom_ms * 1e-3) / 1e12
    line = {
        "metric": "ensemble trajectory-steps/s (256 uneven trajectories, one graph per step)",
        "value": steps_per_s * n,
        "unit": "trajectory-steps/s",
        "n_gpus": 1,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "dtype": "f64" if args.precision == 0 else "f32+f64",
        "data": "synthetic",
        "config": {"workload": f"ensemble: {shapes.count((32, 16, 16))}x(N32,|k|<16,m<16) + "
                               f"{shapes.count((48, 24, 24))}x(N48,|k|<24,m<24) + "
                               f"{shapes.count((64, 32, 32))}x(N64,|k|<32,m<32), "
                               "Re U[1800,2600], amp logU[1e-3,1e-1], dt=0.005",
                   "l2": "working set > L2 (no flush needed)",
                   "autotune": bool(args.autotune)},
        "gdof_steps_per_s": steps_per_s * dofs / 1e9,
        "hbm_roofline_frac": algo_bytes * steps_per_s / (peaks["hbm_gbs"] * 1e9),
        "roofline": {"kernel": dom, "bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                     "frac": ach / pk, "traffic": None, "peak_source": src},
        "setup_s": setup_s,
        "inputs_s": inputs_s,
        "clocks": clk,
        "energy_EID_first_member_of_each_shape": [[float(x) for x in v] for v in E],
    }
    print(json.dumps(line), flush=True)


def large_oracle_check(opf, w):
    """Errors of the large grid against the FP64 oracle where the oracle can
    follow: the nonlinear term of the start (FP64 and mixed precision), and
    one FP64 predictor-only step (n_corr = 0) on sampled modes, whose dense
    solves the oracle affords one by one."""
    import numpy as np

    from oracle.opf_oracle import Oracle, Params
    from paper_1705_03838_gb300 import inputs

    args_h = (w["N"], w["K"], w["M"], w["m_p"], w["alpha"], w["Re"], 2e-5)
    U0 = inputs.workload_state("large")
    t0 = time.time()
    o = Oracle(Params(*args_h))
    Nref = o.nonlinear(U0)
    K = w["K"]
    modes = [(0, K - 1), (0, K), (1, K - 2), (17, K - 34), (64, K + 90), (100, K - 121), (127, 2 * K - 2)]
    sub = o.solve_modes(U0, Nref, modes)
    host_s = time.time() - t0
    h = opf.opf_create(*args_h)
    out = {}
    for prec, name in ((0, "fp64"), (1, "mixed")):
        opf.opf_set_option(h, "precision", prec)
        got = opf.opf_nonlinear(h, U0)
        out[f"nonlinear_{name}_rel_l2"] = float(np.linalg.norm(got - Nref) / np.linalg.norm(Nref))
    opf.opf_set_option(h, "precision", 0)
    opf.opf_set_option(h, "n_corr", 0)
    opf.opf_set_state(h, U0)
    opf.opf_step(h, 1)
    U1 = opf.opf_get_state(h)
    got = np.stack([U1[:, m, kk] for m, kk in modes])
    want = np.stack([sub[mk][0] for mk in modes])
    out["predictor_solve_fp64_rel_l2_on_sampled_modes"] = float(np.linalg.norm(got - want) / np.linalg.norm(want))
    out["sampled_modes_m_kk"] = modes
    out["oracle_host_seconds"] = host_s
    out["note"] = LARGE_ORACLE_NOTE
    opf.opf_destroy(h)
    return out


def run_large(args):
    """Large turbulent-start run, mixed precision: Re=5300, alpha=0.4
    (L = 5 pi R), N=128, |k|<128, m<128, m_p=1, broadband perturbation of
    amplitude 0.3, CFL-controlled dt <= 0.002 (C = 0.5).  Reports steps/s,
    the dt range, the device footprint, and the energy difference from the
    FP64 path over the same dt sequence (first 50 steps)."""
    import torch

    from paper_1705_03838_gb300 import build as _build, inputs, opf

    torch.cuda.set_device(0)
    _build.build()
    w = inputs.WORKLOADS["large"]
    args_h = (w["N"], w["K"], w["M"], w["m_p"], w["alpha"], w["Re"], w["dt"])
    free0, total = torch.cuda.mem_get_info()
    h = opf.opf_create(*args_h)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    stream = torch.cuda.current_stream()
    opf.opf_set_stream(h, stream.cuda_stream)
    U0 = inputs.workload_state("large")
    res = {}
    # FP64 first with CFL control, recording its dt sequence; the mixed run
    # replays the same sequence for its first 50 steps (same time levels),
    # then keeps CFL control on for the timed remainder
    opf.opf_set_option(h, "precision", 0)
    opf.opf_set_state(h, U0)
    opf.opf_set_option(h, "cfl", 0.5)
    opf.opf_set_option(h, "dt_max", w["dt"])
    dts64 = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for i in range(50):
        dts64.append(opf.opf_get_dt(h))
        opf.opf_step(h, 1)
    ev1.record(stream)
    torch.cuda.synchronize()
    res[0] = {"ms_per_step": ev0.elapsed_time(ev1) / 50, "E": opf.opf_energy(h)}
    opf.opf_set_option(h, "cfl", 0.0)
    opf.opf_set_option(h, "precision", 1)
    opf.opf_set_state(h, U0)
    for d in dts64:
        opf.opf_set_option(h, "dt", d)
        opf.opf_step(h, 1)
    E50 = opf.opf_energy(h)
    opf.opf_set_option(h, "cfl", 0.5)
    dts = []
    torch.cuda.synchronize()
    ev0.record(stream)
    for i in range(args.steps):
        opf.opf_step(h, 1)
        dts.append(opf.opf_get_dt(h))
    ev1.record(stream)
    torch.cuda.synchronize()
    res[1] = {"ms_per_step": ev0.elapsed_time(ev1) / args.steps, "steps": args.steps,
              "dt_min": min(dts), "dt_max": max(dts), "E": E50}
    # kernel shares and the dominant kernel's rate from two instrumented steps
    opf.opf_set_option(h, "timing", 1)
    opf.opf_kernel_times(h, reset=True)
    opf.opf_step(h, 2)
    kt = opf.opf_kernel_times(h, reset=True)
    opf.opf_set_option(h, "timing", 0)
    costs = kernel_costs(w, 1)
    per = {k: v[0] / max(1, v[1]) for k, v in kt.items() if v[1] > 0}
    dom = max(per, key=per.get)
    pk, src = kernel_peak(dom, 1)
    ach = costs[dom]["flops"] / (per[dom] * 1e-3) / 1e12
    roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
            "traffic": None, "peak_source": src, "launch_ms": per[dom]}
    opf.opf_destroy(h)
    oracle_err = large_oracle_check(opf, w)
    dof = 3 * w["N"] * (2 * w["K"] - 1) * (2 * w["M"] - 1)
    line = {
        "metric": "large run timesteps/s (CFL-controlled dt, includes per-step dt control)",
        "value": 1000.0 / res[1]["ms_per_step"],
        "unit": "timesteps/s",
        "n_gpus": 1,
        "steps": res[1]["steps"],
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": "large: N=128 |k|<128 m<128 m_p=1 Re=5300 alpha=0.4 amp=0.3, CFL C=0.5, dt<=0.002"},
        "gdof_steps_per_s": dof * 1000.0 / res[1]["ms_per_step"] / 1e9,
        "fp64_timesteps_per_s": 1000.0 / res[0]["ms_per_step"],
        "dt_range_mixed": [res[1]["dt_min"], res[1]["dt_max"]],
        "device_footprint_gb": (free0 - free1) / 1e9,
        "energy_rel_diff_mixed_vs_fp64_after_50_steps": float(abs(res[1]["E"][0] - res[0]["E"][0]) / res[0]["E"][0]),
        "roofline": roof,
        "oracle_error": oracle_err,
        "hbm_roofline_frac": step_algorithmic_bytes(w, 1) * (1000.0 / res[1]["ms_per_step"])
        / (load_peaks()[0]["hbm_gbs"] * 1e9),
    }
    print(json.dumps(line), flush=True)


LEARNED = dict(N=48, K=16, M=16, m_p=2, alpha=1.25, dt=0.005, precision=1,
               Re_train=(2000.0, 2500.0), Re_test=2250.0, amp=(0.03, 0.12), B_train=56, B_val=6, B_test=8,
               seed=1705, warmup=20.0, n_snap=320, every=0.5, T_min=10.0, T_max=100.0, thresh=0.3,
               hidden=384, steps=3000, batch=64, lr=1e-3, lam=1.0, net_seed=5, eval_every=200,
               nk_guesses=12, nk_T_max=16.0,
               nk=dict(max_newton=2, max_krylov=12, max_hook=4, dt=0.005, tol=1e-10))


# The same pipeline on targets the solver certifies: rotating pipe flow
# (frame rotation Omega = 1 U_cl/R about the axis, alpha = 1, m_p = 2), whose
# Hagen-Poiseuille flow loses stability near Re = 108 to a helical mode that
# saturates into a travelling wave; trajectories at Re in [125, 155] from
# seeded perturbations, snapshots of the saturation and the wave, 720 feature
# channels (|k| < 8, m < 8) over 24 radial points.  A travelling wave recurs
# for any T with s = c T, so the Newton problems fix T at the guess's value
# and solve for s (the axial phase condition).
LEARNED_ROT = dict(N=24, K=8, M=8, m_p=2, alpha=1.0, dt=0.01, precision=1, rot=(0.0, 0.0, 1.0),
                   Re_train=(125.0, 155.0), Re_test=140.0, amp=(0.03, 0.12), B_train=56, B_val=6, B_test=8,
                   seed=1705, warmup=60.0, n_snap=320, every=0.5, T_min=2.0, T_max=12.0, thresh=0.3,
                   hidden=384, steps=2000, batch=64, lr=1e-3, lam=1.0, net_seed=5, eval_every=200,
                   nk_guesses=12, nk_T_max=12.0,
                   nk=dict(max_newton=8, max_krylov=30, max_hook=4, dt=0.01, tol=1e-10, fix_T=1, fix_s=0))


def run_learned(args):
    """Learned Newton-Krylov proposals: 64 trajectories (56 for training, 6 of
    them for validation, at Re uniform in [2000, 2500]; 8 held out at Re = 2250)
    of N=48, |k|<16, m<16, m_p=2 (the named resolution with the radial points
    raised from 32 to 48: at N=32 these starts go non-finite whatever K and
    M, at N=48 they stay resolved), 20,480 snapshots every 0.5 time units; the
    BF16 network trained by the library's own kernels; Newton-Krylov-hookstep
    from the 12 best held-out recurrences with recurrence, learned,
    learned-state and snapshot-with-mean-period guesses under the same budget."""
    import torch

    from paper_1705_03838_gb300 import build as _build, learned, opf

    torch.cuda.set_device(0)
    _build.build()
    opf.lib()
    rotating = args.workload == "learned_rot"
    cfg = LEARNED_ROT if rotating else LEARNED
    t0 = time.perf_counter()
    res = learned.run_pipeline(opf, torch, cfg,
                               log=lambda *a: print(*a, f"[{time.perf_counter() - t0:.0f} s]", file=sys.stderr,
                                                    flush=True))
    nk = res.get("nk", {})
    arms = {name: {"certified_fraction": v.get("certified_fraction"),
                   "median_newton_iterations_to_certification": v.get("median_newton_iterations_to_certification"),
                   "median_final": v.get("median_final"), "seconds": v.get("seconds")}
            for name, v in nk.items()}
    if rotating:
        workload = ("learned proposals on certifiable targets: rotating pipe (Omega_z = 1), N=24 |k|<8 m<8 m_p=2 "
                    "alpha=1, Re in [125,155], 64 trajectories x 320 snapshots")
    else:
        workload = ("learned proposals: N=48 |k|<16 m<16 m_p=2 alpha=1.25, Re in [2000,2500], "
                    "64 trajectories x 320 snapshots")
    line = {
        "metric": "Newton-Krylov-hookstep from learned vs recurrence guesses: median final relative residual",
        "value": nk.get("learned", {}).get("median_final"),
        "unit": "relative residual",
        "higher_is_better": False,
        "n_gpus": 1,
        "dtype": "bf16 net (f32 accumulate); f32+f64 snapshots; f64 Newton",
        "data": "synthetic (the solver's own trajectories from seeded perturbations)",
        "config": {"workload": workload},
        "recurrence_median_final": nk.get("recurrence", {}).get("median_final"),
        "snapshot_mean_T_median_final": nk.get("snapshot_mean_T", {}).get("median_final"),
        "arms": arms,
        "details": res,
    }
    print(json.dumps(line, default=float), flush=True)


def run_net(args):
    """Proposal-network training step (the only dense contraction): B=64
    snapshots of 720 channels over L=48 radial points, hidden 384 (2.10 M
    parameters), forward + backward + Adam on the tensor cores.  Reports
    the step time and the GEMM throughput against the measured BF16 peak."""
    import torch

    from paper_1705_03838_gb300 import build as _build, opf

    torch.cuda.set_device(0)
    _build.build()
    opf.lib()
    cin, hid, L, nout, B = 720, 384, 48, 3, 64
    net = opf.opf_net_create(cin, hid, L, nout, seed=1)
    g = torch.Generator().manual_seed(0)
    x = torch.randn(B, L, cin, generator=g).cuda()
    ty = 0.1 * torch.randn(B, L, cin, generator=g).cuda()
    tz = torch.randn(B, nout, generator=g).cuda()
    step = lambda: opf.opf_net_train_step(net, x.data_ptr(), ty.data_ptr(), tz.data_ptr(), B, 1.0, 1e-4)
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1000.0 / args.steps
    F1, F2, F3 = (2.0 * B * L * 3 * cin * hid, 2.0 * B * L * 3 * hid * hid, 2.0 * B * L * 3 * hid * cin)
    flops = 2 * F1 + 3 * F2 + 3 * F3  # forward, weight gradients, input gradients of layers 2 and 3
    peaks, src = load_peaks()
    line = {
        "metric": "proposal-network training steps/s (BF16 tensor-core GEMMs, FP32 accumulate)",
        "value": 1000.0 / ms, "unit": "steps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": f"net: B={B} L={L} channels={cin} hidden={hid} params={opf.opf_net_param_count(net)[0]}"},
        "gemm_tflops_per_step": flops / (ms * 1e-3) / 1e12,
        "bf16_peak_tflops": peaks.get("bf16_tflops"),
        "bf16_peak_source": src,
    }
    print(json.dumps(line), flush=True)


def run_floquet(args):
    """Leading Floquet multipliers of 16 perturbed laminar states (N=32,
    |k|<16, m<16, m_p=2, alpha=1.25, Re=2000), period T=2 at dt=0.01: 30
    Arnoldi steps, each one batched 200-step integration of all 16 states."""
    import numpy as np
    import torch

    from paper_1705_03838_gb300 import build as _build, inputs, opf

    torch.cuda.set_device(0)
    _build.build()
    opf.lib()
    N, K, M, m_p, alpha, Re, T, dt, k, count = 32, 16, 16, 2, 1.25, 2000.0, 2.0, 0.01, 30, 16
    lam = inputs.laminar_state(N, K, M)
    states = [lam + inputs.seeded_state(N, K, M, m_p, alpha, 1e-3, 700 + i, laminar=False) for i in range(count)]
    t0 = time.perf_counter()
    ev, res = opf.opf_floquet(N, K, M, m_p, alpha, Re, states, [T] * count, [0.0] * count, k, 4, dt, precision=0)
    sec = time.perf_counter() - t0
    steps = (k + 1) * int(round(T / dt)) * count
    line = {
        "metric": "Floquet multipliers: batched Arnoldi trajectory-steps/s (FP64 integrations)",
        "value": steps / sec, "unit": "trajectory-steps/s", "n_gpus": 1, "higher_is_better": True,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"floquet: {count} states N={N} |k|<{K} m<{M} m_p={m_p} Re={Re} T={T} dt={dt}, "
                               f"{k} Arnoldi steps"},
        "seconds": sec,
        # Ritz values of largest modulus and their residual estimates: after 30
        # steps on this strongly non-normal map they are not yet converged
        # eigenvalues (large residuals); the line measures the throughput
        "ritz_values_state0": [[float(z.real), float(z.imag)] for z in ev[0]],
        "residual_estimates_state0": [float(r) for r in res[0]],
    }
    print(json.dumps(line), flush=True)


def run_kernels(args):
    """Per-kernel device times of the time step of one workload (option
    timing 1: a CUDA event pair around every kernel of the step graph), after
    two untimed steps: microseconds per launch and launches per kernel, and
    the wall time per step with the events in place.  Small enough to run
    under a profiler (--steps few)."""
    import torch

    from paper_1705_03838_gb300 import build as _build, inputs, opf

    torch.cuda.set_device(0)
    _build.build()
    wl = args.kernels_workload
    w = inputs.WORKLOADS[wl]
    h = opf.opf_create(w["N"], w["K"], w["M"], w["m_p"], w["alpha"], w["Re"], w["dt"])
    opf.opf_set_option(h, "precision", args.precision)
    opf.opf_set_state(h, inputs.workload_state(wl))
    opf.opf_step(h, 2)
    torch.cuda.synchronize()
    opf.opf_set_option(h, "timing", 1)
    opf.opf_kernel_times(h, reset=True)
    t0 = time.time()
    opf.opf_step(h, args.steps)
    torch.cuda.synchronize()
    wall = (time.time() - t0) / args.steps
    kt = opf.opf_kernel_times(h, reset=True)
    line = {
        "metric": "per-kernel device time of the time step (events around every kernel)",
        "unit": "us per launch", "n_gpus": 1, "steps": args.steps, "dtype": "f64" if args.precision == 0 else "f32+f64",
        "data": "synthetic", "config": {"workload": wl, "precision": args.precision},
        "kernels": {k: {"us_per_launch": ms * 1e3 / max(n, 1), "launches": n} for k, (ms, n) in kt.items()},
        "wall_ms_per_step_with_events": wall * 1e3,
        "energy_EID": [float(x) for x in opf.opf_energy(h)],
    }
    print(json.dumps(line), flush=True)


def run_peaks(args):
    """FP64 and FP32 FMA throughput of this GPU (the library's probe kernel:
    independent FMA recurrences over every SM), best of three each, beside
    the unit-count peaks the ALU rooflines use."""
    import torch

    from paper_1705_03838_gb300 import build as _build, opf

    torch.cuda.set_device(0)
    _build.build()
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    f64 = max(opf.opf_fma_rate(0) for _ in range(3))
    f32 = max(opf.opf_fma_rate(1) for _ in range(3))
    clk = clocks.stop()
    line = {
        "metric": "FMA throughput (measured) vs unit-count peaks", "unit": "TFLOP/s", "n_gpus": 1,
        "fp64_measured": f64, "fp32_measured": f32,
        "fp64_unit_count_peak": FP64_PEAK_TFLOPS, "fp32_unit_count_peak": FP32_PEAK_TFLOPS,
        "fp64_frac_of_unit_count": f64 / FP64_PEAK_TFLOPS, "fp32_frac_of_unit_count": f32 / FP32_PEAK_TFLOPS,
        "clocks": clk, "gpu": torch.cuda.get_device_name(0),
    }
    print(json.dumps(line), flush=True)


def run_gpu(args, w):
    import numpy as np
    import torch

    from paper_1705_03838_gb300 import build as _build, inputs, opf

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or not _build.up_to_date():
        _build.build()
    if world > 1:
        dist.barrier()
    stream = torch.cuda.current_stream()
    h = opf.opf_create(w["N"], w["K"], w["M"], w["m_p"], w["alpha"], w["Re"], w["dt"])
    opf.opf_set_stream(h, stream.cuda_stream)
    # each replica runs its own seeded trajectory
    U0 = inputs.seeded_state(w["N"], w["K"], w["M"], w["m_p"], w["alpha"], w["amplitude"],
                             w["seed"] + rank, w["envelope"])
    opf.opf_set_state(h, U0)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    clean = torch.ones(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def flush_l2():
        flush.zero_()  # evicts the step's working set
        clean.sum()    # evicts the flush's dirty lines outside the timed region

    names = ["curl", "zsynth", "product", "zanalysis", "solve"]

    def timed(precision):
        """K steps at one precision from U0; per-step CUDA events, L2 flushed
        between, the step graph free of any inner event record.  A few
        untimed steps with an event pair around every kernel give the kernel
        shares and the dominant kernel; after the timed steps, as many steps
        again with an event pair around the dominant kernel only give its
        live duration."""
        opf.opf_set_option(h, "precision", precision)
        opf.opf_set_state(h, U0)
        for _ in range(args.warmup):
            flush_l2()
            opf.opf_step(h, 1)
        opf.opf_set_state(h, U0)
        opf.opf_set_option(h, "timing", 1)
        opf.opf_kernel_times(h, reset=True)
        for _ in range(max(3, args.warmup)):
            flush_l2()
            opf.opf_step(h, 1)
        kt_all = opf.opf_kernel_times(h, reset=True)
        dom = max(kt_all, key=lambda k: kt_all[k][0])
        opf.opf_set_option(h, "timing", 0)
        opf.opf_step(h, 1)  # capture the plain step graph outside the timed region
        opf.opf_set_state(h, U0)
        clocks = ClockSampler(local)
        clocks.start()
        time.sleep(0.3)
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        wall0 = time.time()
        for i in range(args.steps):
            flush_l2()
            ev0[i].record(stream)
            opf.opf_step(h, 1)
            ev1[i].record(stream)
        torch.cuda.synchronize()
        wall = time.time() - wall0
        if world > 1:
            dist.barrier()
        clk = clocks.stop()
        total = sum(a.elapsed_time(b) for a, b in zip(ev0, ev1))
        # the dominant kernel's live duration: the same steps with an event
        # pair around that kernel only
        opf.opf_set_option(h, "timing", 2)
        opf.opf_set_option(h, "timed_kernel", names.index(dom))
        opf.opf_set_state(h, U0)
        opf.opf_step(h, 1)
        opf.opf_set_state(h, U0)
        opf.opf_kernel_times(h, reset=True)
        for _ in range(args.steps):
            flush_l2()
            opf.opf_step(h, 1)
        kt_live = opf.opf_kernel_times(h, reset=True)
        opf.opf_set_option(h, "timing", 0)
        # per-launch averages (every kernel launches twice per step): shares
        # from the instrumented steps, the dominant kernel's from the steps
        # that time it alone
        kt = {k: (v[0] / max(1, v[1]), 1) for k, v in kt_all.items()}
        kt[dom] = (kt_live[dom][0] / max(1, kt_live[dom][1]), 1)
        energy = opf.opf_energy(h)
        total = max_over_ranks(total, dist, "cuda")
        return total, kt, clk, wall, energy

    res = {}
    for prec in (0, 1):
        res[prec] = timed(prec)
    total_ms, ktimes, clk, wall, E = res[args.precision]
    E64, E32 = res[0][4], res[1][4]

    # end-to-end through the public API with host buffers: per step, copy the
    # state in from pinned memory, advance one step and copy the new state
    # (the step's result) out to pinned memory.  E, I, D (a diagnostic with an
    # FP64 curl of its own) are read once after the loop.
    opf.opf_set_option(h, "precision", args.precision)
    pinned = torch.from_numpy(U0.view(np.float64).copy()).pin_memory()
    pinned_out = torch.empty_like(pinned).pin_memory()
    e2e_steps = max(3, min(args.steps, 50))
    opf.opf_step(h, 1)
    torch.cuda.synchronize()
    t0 = time.time()
    for _ in range(e2e_steps):
        opf.lib().opf_set_state(h.ptr, pinned.data_ptr())
        opf.opf_step(h, 1)
        opf.lib().opf_get_state(h.ptr, pinned_out.data_ptr())
    torch.cuda.synchronize()
    e2e_s = time.time() - t0
    E = opf.opf_energy(h)
    e2e_state_ok = bool(np.isfinite(pinned_out.numpy()).all())
    e2e_rate = job_rate(e2e_steps, world, max_over_ranks(e2e_s, dist, "cuda"))

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    value = job_rate(args.steps, world, total_ms / 1000.0)
    peaks, peak_kind = load_peaks()
    def roofline(kt, precision):
        costs = kernel_costs(w, precision)
        dom = max(kt, key=lambda k: kt[k][0])
        dom_ms = kt[dom][0] / max(1, kt[dom][1])
        pk, src = kernel_peak(dom, precision)
        ach = costs[dom]["flops"] / (dom_ms * 1e-3) / 1e12
        traffic = PROFILED_DRAM_BYTES.get((dom, precision))
        return {"kernel": dom, "bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                "frac": ach / pk, "traffic": traffic,
                "traffic_source": PROFILE_FILES.get(dom) if traffic is not None else None,
                "peak_source": src, "launch_ms": dom_ms}

    roof = roofline(ktimes, args.precision)
    fp64_value = job_rate(args.steps, world, res[0][0] / 1000.0)
    mixed_value = job_rate(args.steps, world, res[1][0] / 1000.0)
    hbm_frac = step_algorithmic_bytes(w, args.precision) * value / world / (peaks["hbm_gbs"] * 1e9)

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        sps, n, setup, secs = oracle_timing(seconds_budget=15.0)
        agg, nproc, nall = oracle_timing_all_cores(seconds_budget=10.0)
        small = oracle_small_full()
        cpu = {"value": agg, "unit": "timesteps/s", "cores": nproc, "kind": "oracle",
               "sample": f"{nproc} single-threaded oracle processes on {nproc} host cores, each stepping its own "
                         f"seeded trajectory of the same workload for ~10 s after 1 setup step ({nall} steps "
                         f"in all); value = the sum of their step rates",
               "host_cores": os.cpu_count(),
               "single_thread": {"value": sps, "unit": "timesteps/s", "cores": 1,
                                 "sample": f"{n} full oracle steps of the same workload after 1 setup step "
                                           f"({setup:.1f} s), {secs:.1f} s"},
               "small_workload_100_steps": {"seconds": small["seconds"], "cores": 1,
                                            "timesteps_per_s": 100.0 / small["seconds"]},
               "large_workload": LARGE_ORACLE_NOTE}
    # per pass: curl + 3 transform kernels + solve (mixed); FP64 steps take
    # the curl inside the solve
    launches_per_step = (5 if args.precision == 1 else 4) * 2
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "timesteps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if args.precision == 0 else "f32+f64",
        "precision_compare": {
            "fp64": {"value": fp64_value, "ms_per_step": res[0][0] / args.steps,
                     "roofline": roofline(res[0][1], 0)},
            "mixed": {"value": mixed_value, "ms_per_step": res[1][0] / args.steps,
                      "roofline": roofline(res[1][1], 1)},
            "mixed_over_fp64": mixed_value / fp64_value,
            "mixed_energy_rel_err_vs_fp64_after_steps": float(abs(E32[0] - E64[0]) / E64[0]),
        },
        "data": "synthetic",
        "config": config_dict(w, args.precision),
        "gdof_steps_per_s": value * dof(w) / 1e9,
        "hbm_roofline_frac": hbm_frac,
        "hbm_peak_gbs": peaks["hbm_gbs"],
        "hbm_peak_source": peak_kind,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_rate, "unit": "timesteps/s",
                "h2d_bytes_per_step": int(U0.nbytes), "d2h_bytes_per_step": int(U0.nbytes),
                "per_step": "set_state from pinned host memory, one step, get_state (the new state) to "
                            "pinned host memory", "state_finite": e2e_state_ok},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
        "wall_s_timed_region": wall,
        "energy_EID": [float(x) for x in E],
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--precision", type=int, default=1,
                    help="headline precision: 1 = mixed (default), 0 = FP64; both are timed")
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="medium",
                    choices=["medium", "ensemble", "large", "learned", "learned_rot", "net", "floquet", "kernels", "peaks"],
                    help="medium: the default single-run line; ensemble: the batched workload; large: the "
                         "CFL-controlled large run; learned: the learned Newton-Krylov proposal pipeline; learned_rot: the "
                         "same pipeline on the travelling waves of rotating pipe flow (certifiable targets); "
                         "net: the proposal network's training step; floquet: batched Arnoldi "
                         "Floquet multipliers; kernels: per-kernel device times of one workload's step "
                         "(--kernels-workload, --precision, --steps); peaks: measured FP64/FP32 FMA rates")
    ap.add_argument("--kernels-workload", default="medium",
                    help="workload of --workload kernels: small, medium or large")
    ap.add_argument("--autotune", type=int, default=0)
    ap.add_argument("--ens-count", type=int, default=256,
                    help="trajectories of --workload ensemble (256 = the full workload; fewer, in the same "
                         "proportions, for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    w = workload_params()
    if args.impl == "reference":
        run_reference(args, w)
    elif args.workload == "ensemble":
        run_ensemble(args)
    elif args.workload == "large":
        run_large(args)
    elif args.workload in ("learned", "learned_rot"):
        run_learned(args)
    elif args.workload == "net":
        run_net(args)
    elif args.workload == "floquet":
        run_floquet(args)
    elif args.workload == "kernels":
        run_kernels(args)
    elif args.workload == "peaks":
        run_peaks(args)
    else:
        run_gpu(args, w)


if __name__ == "__main__":
    main()
