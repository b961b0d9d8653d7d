#!/usr/bin/env python
"""Throughput of the GB300 ICON-type dycore step on R2B6 L90.

Workload (the configuration the headline metric is quoted on): icosahedral
R2B6 grid (327 680 cells, 491 520 edges), 90 levels to 30 km, dt = 360 s,
5 dynamical substeps + diffusion per step, Rayleigh damping above 20 km,
balanced JW-type baroclinic jet with the seeded Gaussian perturbation
(seed 2).  Synthetic inputs (no dataset exists in this environment).

A "step" is one full dycore time step.  The device-resident legs time K
steps replayed as one CUDA graph each, with CUDA events on the stream the
library launches on; the state (1.5 GB) is larger than L2, so no flush is
needed.  Legs: FP64 (the headline value); mixed precision (FP32 stencils,
double-word FP32 column solve); mixed with an FP64 column solve; mixed plus
the learned corrector (trained on the GPU first, untimed, on other seeds:
steps with 3 substeps plus the learned increments, the check and any
fallback to the plain step).  After its timed steps every leg runs on,
untimed, to one simulated day (240 steps), where the surface pressure and
the 850 hPa temperature are compared with the FP64 leg's.  The end-to-end
leg calls the C-ABI with HOST arrays: the library copies the state in and
out around every step.  The mountain section runs the R2B7 L90 Gaussian-
mountain configuration (dt 180 s, terrain-following heights) in FP64, mixed
and mixed + learned.  N>1 (torchrun) runs N independent replicas (ensemble
members), one per GPU.

``--impl reference`` times the FP64 CPU oracle instead (on the host cores),
each step a bounded sample: one substep and one diffusion call on R2B4 L90,
extrapolated to a full R2B6 L90 step (x5 substeps, x16 cells).
"""
import argparse
import gc
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(bisections=6, nlev=90, dtime=360.0, ndyn=5, seed=2, rayleigh=0.05)
# the mountain configuration: Gaussian mountain 2 km high, 1500 km e-folding radius
MOUNTAIN = dict(bisections=7, nlev=90, dtime=180.0, ndyn=5, seed=3, rayleigh=0.05, h0=2000.0, d=1.5e6,
                max_steps=10)
SAMPLE_BISECTIONS = 4          # reference / cpu_baseline sample grid (1/16 of the R2B6 columns)
METRIC = "dycore steps/s + HBM GB/s fraction at R2B6 L90: FP64 vs mixed+learned"
FP64_PEAK_TFLOPS = 1.25        # nominal GB300 FP64 (152 SMs x 2 DFMA/clk x 2 flop x ~2.06 GHz)
HBM_FALLBACK_GBS = 6800.0      # used only when the measured peaks are absent


def hbm_peak():
    """(GB/s, source): the measured copy bandwidth, else the fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return HBM_FALLBACK_GBS, "fallback"


# FP64 flops per unit (FMA = 2, add/mul = 1, a reciprocal = its FP64 add and
# two FMAs), counted from the arithmetic each kernel evaluates; the unit is
# one (point, level).  va_cell_vert: the mean of its predictor and corrector
# forms per unit of its combined cell and vertex launch.
FLOPS_PER_UNIT = {
    "va_edge_pre": 15, "va_cell_vert": 14, "va_edge_tend": 21, "va_cell_w": 11,
    "sn_cell_grad": 32, "sn_edge_pred": 24, "sn_cell_div": 5, "sn_cell_fluxdiv": 27,
    "sn_edge_flux": 6, "sn_cell_fluxsum": 12,
    "sn_column_pred": 83, "sn_edge_corr": 11, "sn_column_corr": 84,
    "diff_div_curl_uv": 30, "diff_edge_smag": 46, "diff_second": 30,
    "diff_edge_update": 12, "diff_cell_update": 12, "va_concorr": 20,
}

SUFFIXES = ("_f32", "_terrain", "_mx64", "_mx")


def base_name(name):
    """The kernel a launch name belongs to: without the precision and terrain suffixes."""
    changed = True
    while changed:
        changed = False
        for s in SUFFIXES:
            if name.endswith(s):
                name, changed = name[:-len(s)], True
    return name


def units_per_launch(name, nc, ne, nv, nlev):
    full = {"c": nc * nlev, "e": ne * nlev, "v": nv * nlev}
    half = {"c": nc * (nlev + 1), "e": ne * (nlev + 1), "v": nv * (nlev + 1)}
    return {
        "va_edge_pre": full["e"], "va_cell_vert": full["c"] + half["v"], "va_edge_tend": half["e"],
        "va_cell_w": half["c"], "va_concorr": half["c"], "sn_cell_grad": full["c"], "sn_edge_pred": full["e"],
        "sn_column_pred": full["c"], "sn_edge_corr": full["e"], "sn_column_corr": full["c"],
        "sn_cell_div": full["c"], "sn_cell_fluxdiv": full["c"], "sn_edge_flux": full["e"],
        "sn_cell_fluxsum": full["c"],
        "diff_div_curl_uv": full["c"] + full["v"], "diff_edge_smag": full["e"],
        "diff_second": half["c"] + full["v"], "diff_edge_update": full["e"], "diff_cell_update": half["c"],
        "mx_refresh": full["e"] + half["c"], "lc_col_inputs": full["c"], "lc_edge_inputs": full["e"],
        "va_fused": half["c"],  # rows A1-A4 over cell patches: per cell and half level
    }[base_name(name)]


def state_bytes(nc, ne, nlev):
    return 8 * (ne * nlev + nc * (nlev + 1) + 4 * nc * nlev)


# Compulsory HBM bytes of one step: every prognostic (vn, w, rho, exner,
# theta_v, exner_pr) read and written once per substep, plus once more for
# the diffusion.
def compulsory_bytes_per_step(nc, ne, nlev, ndyn):
    return 2 * state_bytes(nc, ne, nlev) * (ndyn + 1)


def stage_bytes_per_step(leg, nc, ne, nv, nlev, ndyn):
    """Algorithmic bytes of one step: every field each kernel reads or writes,
    counted once per launch (the stage boundaries of the kernel plan).
    Stencil fields are FP64 (leg fp64) or FP32 (leg mixed); the state, the
    exner history, the extrapolated exner perturbation, the flux divergences
    and the column solve's scratch are 8 bytes in both.  None for the learned
    leg (its networks' traffic depends on the batch chunking)."""
    if leg not in ("fp64", "mixed"):
        return None
    mixed = leg == "mixed"
    s = 4 if mixed else 8
    E, Eh, C, Ch = ne * nlev, ne * (nlev + 1), nc * nlev, nc * (nlev + 1)
    V, Vh = nv * nlev, nv * (nlev + 1)
    va = (2 * 3 * E * s                                                    # va_edge_pre, pred + corr
          + (2 * E + C + V + Ch + Vh) * s + (2 * E + 3 * C + V + Ch + Vh) * s  # va_cell_vert (corr: + div damping)
          + 2 * (3 * E + Eh + Ch + C + V + Vh) * s                         # va_edge_tend
          + 2 * (2 * Ch + Eh) * s)                                         # va_cell_w
    sn = (6 * C * s + 3 * C * 8                                           # sn_cell_grad (+ exner, history, pex)
          + (7 * E + 6 * C) * s + 8 * C                                    # sn_edge_pred
          + (E + C) * s + 16 * C + (E + C) * s                             # sn_cell_div, pred (+ history) and corr
          + 2 * ((3 * E + C) * s + 16 * C)                                 # sn_cell_fluxdiv
          + 16 * E + (3 * E + C) * s + (4 * E if mixed else 0)             # sn_edge_corr (FP64 vn in place)
          + ((200 + 236) if mixed else (208 + 232)) * C)                   # column solve pred + corr
    diff = ((E + C + 4 * V) * s + (4 * V + C + 2 * E) * s + (2 * E + 2 * Ch + 3 * C + V) * s
            + 16 * E + (2 * E + C + V) * s + (4 * E if mixed else 0)
            + (Ch + C) * s + 16 * Ch + 32 * C + ((4 * Ch + 4 * C) if mixed else 0))
    refresh = (E + Ch + 2 * C) * 12 if mixed else 0                       # mx_refresh
    return ndyn * (va + sn) + diff + refresh


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows if len(r) >= 9 for i in range(4)
                          if r[5 + i].strip().lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def init_ranks(world, backend="nccl"):
    """One process per GPU (replicas): join the process group when world > 1
    (NCCL on the GPUs; gloo in the CPU tests of this logic)."""
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend, init_method="env://")


def max_over_ranks(ms, world, device):
    """The longest of the ranks' timed regions: the job ends with its slowest
    rank, so the whole-job throughput is measured against that time."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, steps, ms):
    """Whole-job steps/s: every rank advances its own replica by `steps` in at
    most `ms` milliseconds (weak scaling: the work per GPU is fixed)."""
    return world * steps / (ms / 1000.0)


def oracle_sample(bisections, nlev, reps, threads=1):
    """Time the oracle (as it stands) on one substep and one diffusion call of
    the given grid, in a fresh process whose numpy/BLAS may use `threads`
    threads; returns [(substep s, diffusion s)] per repetition."""
    code = r"""
import sys, time, json
sys.path.insert(0, %r)
from icon_inputs import make_grid, make_vct, jw_type_state
from oracle import Dycore, DycoreParams
g = make_grid(%d); z = make_vct(%d)
d = Dycore(g, z, DycoreParams(dtime=%r, ndyn_substeps=%d, rayleigh_coeff=%r))
st = jw_type_state(g, z, seed=%d); st['exner_pr'] = d.initial_exner_pr(st['exner'])
out = []
for _ in range(%d):
    t0 = time.perf_counter(); s1 = d.substep(st); t1 = time.perf_counter(); d.diffusion(s1); t2 = time.perf_counter()
    out.append((t1 - t0, t2 - t1))
print(json.dumps(out))
""" % (ROOT, bisections, nlev, WORKLOAD["dtime"], WORKLOAD["ndyn"], WORKLOAD["rayleigh"], WORKLOAD["seed"], reps)
    n = str(threads)
    env = dict(os.environ, OMP_NUM_THREADS=n, OPENBLAS_NUM_THREADS=n, MKL_NUM_THREADS=n, CUDA_VISIBLE_DEVICES="")
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if p.returncode != 0:
        raise RuntimeError(p.stderr)
    return json.loads(p.stdout.strip().splitlines()[-1])


def sample_to_steps_per_s(t_sub, t_diff, scale):
    return 1.0 / (scale * (WORKLOAD["ndyn"] * t_sub + t_diff))


def host_cores():
    return os.cpu_count() or 1


def cpu_baseline(nlev):
    """The numpy oracle on the host cores: one substep + one diffusion on R2B4
    L90, scaled to an R2B6 L90 step; once with every core available to numpy
    and its BLAS (the reported value), once on one thread."""
    scale = 4 ** (WORKLOAD["bisections"] - SAMPLE_BISECTIONS)
    out = {}
    for threads in (host_cores(), 1):
        t_sub, t_diff = oracle_sample(SAMPLE_BISECTIONS, nlev, 1, threads)[0]
        out[threads] = (sample_to_steps_per_s(t_sub, t_diff, scale), t_sub, t_diff)
    v_all, s_all, d_all = out[host_cores()]
    v_one, s_one, d_one = out[1]
    return {"value": v_all, "unit": "steps/s", "cores": host_cores(), "kind": "oracle",
            "sample": "one substep (%.1f s) + one diffusion (%.1f s) of the numpy FP64 oracle on R2B4 L90 "
                      "(1/16 of the R2B6 columns) with %d threads allowed to numpy/BLAS (its element-wise "
                      "arithmetic runs on one core), scaled to an R2B6 L90 step as 16 x (5 substeps + diffusion)"
                      % (s_all, d_all, host_cores()),
            "extrapolated": True,
            "single_thread": {"value": v_one, "cores": 1, "substep_s": s_one, "diffusion_s": d_one}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    nlev = WORKLOAD["nlev"]
    reps = args.warmup + args.steps
    cores = host_cores()
    t0 = time.perf_counter()
    samples = oracle_sample(SAMPLE_BISECTIONS, nlev, reps, cores)[args.warmup:]
    wall = time.perf_counter() - t0
    scale = 4 ** (WORKLOAD["bisections"] - SAMPLE_BISECTIONS)
    step_s = [scale * (WORKLOAD["ndyn"] * a + b) for a, b in samples]
    total = sum(step_s)
    value = args.steps / total
    sample = ("per step: one substep + one diffusion of the numpy FP64 oracle on R2B4 L90, extrapolated x16 "
              "(cells) and x5 (substeps) to an R2B6 L90 step; measured %.1f s of oracle work for %d sample steps"
              % (sum(a + b for a, b in samples), args.steps))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_dict("fp64"),
        "extrapolated": True, "sample_wall_s": wall,
        "cpu_baseline": {"value": value, "unit": "steps/s", "cores": cores, "kind": "oracle", "sample": sample,
                         "extrapolated": True},
        "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def config_dict(prec):
    w = WORKLOAD
    nc = 80 * 4 ** w["bisections"]
    return {"workload": "R2B%d L90 (%d cells, %d edges), dt=%gs, %d substeps + diffusion, %s, "
                        "JW-type jet seed %d" % (w["bisections"], nc, 3 * nc // 2, w["dtime"], w["ndyn"],
                                                 prec.upper(), w["seed"]),
            "grid": "R2B%d" % w["bisections"], "nlev": w["nlev"], "dtime_s": w["dtime"], "ndyn_substeps": w["ndyn"],
            "precision": prec, "cuda_graph": True,
            "l2": "inputs larger than L2 (FP64 state 1.5 GB, scratch ~9 GB); no flush"}


# ---------------------------------------------------------------------------
# DRAM traffic per unit of every kernel, from one-kernel ncu captures
# (dram__bytes_read.sum + dram__bytes_write.sum of one launch, -c 1; the
# column solve's predictor and corrector -c 2) at R2B5 L90 inside the leg's
# timed steps, divided by the units (point-levels) of that launch; scaled to
# the bench's grid by the units per launch.  Kernels that run in row chunks
# (the learned step's networks and increments) carry bytes per unit of a
# whole step instead (PER_STEP_UNITS).  Valid while the sources that define
# the timed kernels are the ones captured (SHA-256 over KERNEL_SOURCES).
DRAM_PER_UNIT = {
    "sources_sha256": "1c755f8073d4233f8d10e6c746013f70051ad72effbae2380259e228a05b1090",
    "bisections": 5, "nlev": 90,
    "legs": {
        "fp64": {
            "diff_cell_update": 57.627, "diff_div_curl_uv": 29.152, "diff_edge_smag": 30.742,
            "diff_edge_update": 38.763, "diff_second": 52.87, "sn_cell_div": 31.13, "sn_cell_fluxsum": 36.227,
            "sn_cell_grad": 66.955, "sn_column_corr": 274.264, "sn_column_pred": 208.707, "sn_edge_corr": 44.137,
            "sn_edge_flux": 42.929, "sn_edge_pred": 92.494, "va_cell_vert": 41.95, "va_cell_w": 25.65,
            "va_edge_pre": 27.746, "va_edge_tend": 51.936},
        "mixed": {
            "diff_cell_update": 56.156, "diff_div_curl_uv": 10.468, "diff_edge_smag": 13.727,
            "diff_edge_update": 28.821, "diff_second": 24.801, "mx_refresh": 20.004, "sn_cell_div": 20.767,
            "sn_cell_fluxdiv": 34.433, "sn_cell_grad": 42.77, "sn_column_corr": 304.048, "sn_column_pred": 201.923,
            "sn_edge_corr": 31.213, "sn_edge_pred": 47.884, "va_cell_vert": 20.033, "va_cell_w": 11.302,
            "va_edge_pre": 11.198, "va_edge_tend": 24.854, "va_fused": 44.53},
        # the learned step: the mixed kernels (their R2B5 figures) and its own
        "learned": {
            "diff_cell_update": 56.156, "diff_div_curl_uv": 10.468, "diff_edge_smag": 13.727,
            "diff_edge_update": 28.821, "diff_second": 24.801, "lc_apply_col": 20.923, "lc_apply_edge": 15.437,
            "lc_col_inputs": 61.505, "lc_edge_inputs": 39.974, "lc_reduce_status": 527360.0,
            "lc_reduce_status2": 9728.0, "mlp_gemm_tc": 12979.303, "mx_refresh": 20.004, "sn_cell_div": 20.767,
            "sn_cell_fluxdiv": 34.433, "sn_cell_grad": 42.77, "sn_column_corr": 304.048, "sn_column_pred": 201.923,
            "sn_edge_corr": 31.213, "sn_edge_pred": 47.884, "va_cell_vert": 20.033, "va_cell_w": 11.302,
            "va_edge_pre": 11.198, "va_edge_tend": 24.854},
    }}

# The files whose code runs on the device in the timed steps.
KERNEL_SOURCES = ("kernels_stencil.cu", "kernels_column.cu", "column_kernel.cuh", "kernels_column_terrain.cu",
                  "kernels_diag.cu", "mlp.cu", "learned.cu", "dfloat.cuh", "kernels.h", "internal.h")


def per_step_units(name, nc, ne, nlev):
    """Units of a whole step of the kernels that run in row chunks, or None:
    the networks' GEMMs (both networks' rows scale with the cells), the
    increments of the column and edge networks, the check's reductions."""
    return {"mlp_gemm_tc": nc, "lc_apply_col": nc * (3 * nlev - 1), "lc_apply_edge": ne * nlev,
            "lc_reduce_status": 1, "lc_reduce_status2": 1}.get(name)


def sources_sha256():
    """sha256 over the library sources that define the timed kernels."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        h.update(name.encode())
        with open(os.path.join(ROOT, "paper_2608_21150_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def dram_table(leg, nlev):
    """Bytes per unit of every kernel of a leg, or None when the captured
    sources or level count differ from the ones running."""
    t = DRAM_PER_UNIT
    if not t["legs"].get(leg) or t["nlev"] != nlev or sources_sha256() != t["sources_sha256"]:
        return None
    return t["legs"][leg]


def dram_measured(leg, prof, nsteps, ms_per_step, sizes, nlev, ndyn):
    """Measured DRAM bytes of a step (per-unit captures x the step's launches
    and units) over the live step time: achieved HBM GB/s, its fraction of the
    measured peak, and the amplification over the algorithmic stage bytes.
    None if a kernel of the step has no captured figure."""
    tab = dram_table(leg, nlev)
    if tab is None:
        return None
    nc, ne, nv = sizes
    total = 0.0
    for k, (n, _) in prof.items():
        b = base_name(k)
        if b not in tab:
            return None
        u = per_step_units(b, nc, ne, nlev)
        total += tab[b] * (u * nsteps if u is not None else units_per_launch(k, nc, ne, nv, nlev) * n)
    b = total / nsteps
    peak, src = hbm_peak()
    gbs = b / (ms_per_step / 1000.0) / 1e9
    stage = stage_bytes_per_step(leg, nc, ne, nv, nlev, ndyn)
    return {"bytes_per_step": b, "achieved_gbs": gbs, "peak_gbs": peak, "peak_source": src, "frac": gbs / peak,
            "stage_bytes_per_step": stage, "amplification": b / stage if stage else None,
            "note": "per-kernel DRAM bytes per unit from one-launch ncu captures at R2B%d L%d, times the units "
                    "and launches of this step, over the event-timed step; of %s peak"
                    % (DRAM_PER_UNIT["bisections"], DRAM_PER_UNIT["nlev"], src)}


# FP64 instructions per unit (DADD + DMUL + DFMA) where ncu counted them
# (`smsp__sass_thread_inst_executed_op_{dadd,dmul,dfma}_pred_on`, R2B5 L90, the
# sources of DRAM_PER_UNIT): the FP64 pipe issues one of any kind per slot, so
# the instruction rate against the pipe's (half the FMA flop rate) is how busy
# the pipe is, whatever the mix of adds and FMAs.
FP64_INSTR_PER_UNIT = {"sn_column_pred": 59.1, "sn_column_corr": 60.0}

# The column solve's predictor and corrector launches are one kernel (one
# function, two forms); the roofline treats them together.
FAMILY = {"sn_column_pred": "sn_column", "sn_column_corr": "sn_column"}


def roofline(prof, nc, ne, nv, nlev, leg="fp64"):
    """FP64-ALU roofline of the kernel family with the largest share of the
    step, with its HBM fraction from the captured bytes per unit."""
    fam = {}
    for k, (n, ms) in prof.items():
        b = base_name(k)
        f = FAMILY.get(b, b)
        units = units_per_launch(k, nc, ne, nv, nlev) * n
        a = fam.setdefault(f, [0, 0.0, 0.0, 0.0, []])
        a[0] += n
        a[1] += ms
        a[2] += FLOPS_PER_UNIT.get(b, 0) * units
        a[3] += units
        a[4].append(b)
    name, (n, ms, flops, units, members) = max(fam.items(), key=lambda kv: kv[1][1])
    achieved = flops / (ms / 1000.0) / 1e12
    issue = None
    if all(m in FP64_INSTR_PER_UNIT for m in members):
        instr = sum(FP64_INSTR_PER_UNIT[base_name(k)] * units_per_launch(k, nc, ne, nv, nlev) * prof[k][0]
                    for k in prof if FAMILY.get(base_name(k), base_name(k)) == name)
        rate = instr / (ms / 1000.0) / 1e12
        issue = {"achieved": rate, "peak": FP64_PEAK_TFLOPS / 2, "unit": "T FP64 instructions/s",
                 "frac": rate / (FP64_PEAK_TFLOPS / 2),
                 "note": "DADD + DMUL + DFMA per unit from ncu counters x units / event time, against the FP64 "
                         "pipe's instruction rate"}
    tab = dram_table(leg, nlev)
    traffic, hbm = None, None
    if tab is not None and all(m in tab for m in members):
        byts = sum(tab[base_name(k)] * units_per_launch(k, nc, ne, nv, nlev) * prof[k][0]
                   for k in prof if FAMILY.get(base_name(k), base_name(k)) == name)
        traffic = byts / n
        peak, src = hbm_peak()
        gbs = byts / (ms / 1000.0) / 1e9
        hbm = {"achieved_gbs": gbs, "peak_gbs": peak, "frac": gbs / peak, "peak_source": src}
    return {"bound": "alu", "kernel": name, "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic, "hbm": hbm, "fp64_issue": issue,
            "note": "FP64 algorithmic flops per launch / event-timed launch duration (CUDA events around every "
                    "launch on the library's stream); peak = nominal FP64 rate from unit counts and clock "
                    "(1.2 TFLOP/s measured by a DFMA probe); traffic = DRAM bytes per launch from the one-kernel "
                    "ncu captures, scaled by units; hbm = that traffic over the event time"}


def kernel_table(prof, nsteps):
    tot = sum(v[1] for v in prof.values()) / nsteps
    return {k: {"launches_per_step": n // nsteps, "ms_per_step": round(m / nsteps, 3),
                "share": round(m / nsteps / tot, 4)} for k, (n, m) in sorted(prof.items(), key=lambda kv: -kv[1][1])}


PRECISIONS = {"fp64": "ICON_PREC_FP64", "mixed": "ICON_PREC_MIXED", "mixed_f64col": "ICON_PREC_MIXED_F64COL"}


def leg_params(P, wl, leg, stream, **over):
    d = dict(dtime=wl["dtime"], ndyn_substeps=wl["ndyn"], rayleigh_coeff=wl["rayleigh"],
             precision=getattr(P, PRECISIONS[leg]), use_graph=1, synchronous=0, stream=stream.cuda_stream,
             fused_advection=int(wl.get("fused_advection", 0)))
    d.update(over)
    return d


def timed_steps(step, n, dev, world, stream, label):
    """n calls of step() between CUDA events on the library's stream, with
    nvidia-smi clock samples; returns (ms over the ranks, clocks)."""
    import torch
    import torch.distributed as dist
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(dev.index)
    sampler.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    torch.cuda.nvtx.range_push(label + "_timed")   # marks the timed steps for profiler filters
    e0.record(stream)
    for _ in range(n):
        step()
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    if world > 1:
        dist.barrier()
    return max_over_ranks(ms, world, dev), clocks


def final_diagnostics(P, D, t, nc, dev):
    import torch
    ps = torch.empty(nc, dtype=torch.float64, device=dev)
    t850 = torch.empty_like(ps)
    try:
        D.diagnostics(t, ps, t850)
        finite = True
    except P.IconError:
        finite = False
    return finite, ps.cpu().numpy(), t850.cpu().numpy()


def measure(P, G, z, st0, leg, args, dev, world, total_steps, wl, nsteps, prof_steps=3, prepare=None):
    """Time nsteps steps of one precision mode (after the warm-up), profile
    prof_steps more kernel by kernel, then run on untimed to total_steps
    steps in all; returns the numbers and the diagnostics at the end.
    prepare(D, st0): completes the initial state from the new dycore."""
    import torch
    stream = torch.cuda.current_stream(dev)
    D = P.Dycore(G, z, leg_params(P, wl, leg, stream))
    if prepare is not None:
        prepare(D, st0)
    t = {k: torch.from_numpy(v).to(dev) for k, v in st0.items()}
    for _ in range(args.warmup):
        D.step(t)
    ms, clocks = timed_steps(lambda: D.step(t), nsteps, dev, world, stream, leg)
    prof = D.profile(t, prof_steps)
    done = args.warmup + nsteps + prof_steps
    for _ in range(max(0, total_steps - done)):
        D.step(t)
    finite, ps, t850 = final_diagnostics(P, D, t, G.n_cells, dev)
    out = dict(ms=ms, clocks=clocks, finite=finite, ps=ps, t850=t850, prof=prof, nsteps_prof=prof_steps,
               launch_config=D.launch_config(), steps_run=max(total_steps, done))
    D.close()
    del t
    return out


def rms_area(area, d):
    import numpy as np
    return float(np.sqrt(np.sum(area * d ** 2) / np.sum(area)))


# The reduced step of the learned leg: 3 substeps instead of 5, with the exner
# extrapolation off and a stronger fourth-order divergence damping (the
# forward-backward substep with extrapolation factor 1/3 is unstable at the
# longer substep; measured on R2B6 L90 at 360 s: with the default scheme 3
# substeps blow up within 8 steps and 2 within 5; with the extrapolation off
# 3 substeps run clean, 2 still blow up at every damping tried).
LEARNED = dict(ndyn_reduced=3, reduced_scheme=dict(exner_exfac=0.0, divdamp_fac=0.004), hidden=512,
               max_batch=262144, train_seeds=(100, 101, 102, 103), spinup=1, snapshots=8, every=3, rows=8192,
               adam_steps=1500, batch=4096, lr=1e-3, max_norm=3.0)


def learned_leg(P, G, z, grid, st0, args, dev, world, f64_final, wl, total_steps, nsteps, ex_ref):
    """Mixed precision + learned corrector: a step with ndyn_reduced substeps,
    the column and edge networks' increments, the norm/finiteness check and the
    plain-step fallback (icon_dycore_step_learned).  The corrector is trained
    first on the GPU (untimed) from paired reduced/plain steps of other seeds
    on the same grid and heights; ex_ref is the reference exner (per level, or
    per column over terrain) for the training states' exner history."""
    import numpy as np
    import torch
    from paper_2608_21150_gb300 import corrector as C
    from icon_inputs import jw_type_state
    L = LEARNED
    nlev = wl["nlev"]
    stream = torch.cuda.current_stream(dev)
    R = P.Dycore(G, z, leg_params(P, wl, "mixed", stream, ndyn_substeps=L["ndyn_reduced"], **L["reduced_scheme"]))
    Pl = P.Dycore(G, z, leg_params(P, wl, "mixed", stream))
    t0 = time.perf_counter()
    gen = torch.Generator()
    gen.manual_seed(0)
    data = C.Dataset()
    for seed in L["train_seeds"]:
        s0 = jw_type_state(grid, z, seed=seed)
        s0["exner_pr"] = s0["exner"] - ex_ref
        st = {k: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k, v in s0.items()}
        for _ in range(L["spinup"]):
            Pl.step(st)
        for _ in range(L["snapshots"]):
            st = C.add_pair(R, Pl, st, data, rows=L["rows"], gen=gen)
            for _ in range(L["every"] - 1):
                Pl.step(st)
        del st
    cx, cy, ex, ey = data.cat()
    del data
    cn, en = C.make_nets(nlev, hidden=L["hidden"], max_batch=L["max_batch"], seed=1)
    lc = C.fit(cn, cx, cy, nlev, L["adam_steps"], batch=L["batch"], lr=L["lr"])
    le = C.fit(en, ex, ey, nlev, L["adam_steps"], batch=L["batch"], lr=L["lr"])
    del cx, cy, ex, ey
    torch.cuda.synchronize(dev)
    train_s = time.perf_counter() - t0

    t = {k: torch.from_numpy(v).to(dev) for k, v in st0.items()}
    fallbacks_warm = 0
    for _ in range(args.warmup):
        fb, _ = P.step_learned(R, Pl, cn, en, t, L["max_norm"])
        fallbacks_warm += int(fb)
    # held-out error of the corrector at the bench state (reduced and learned vs the plain step);
    # a branch from the state, which goes on from t unchanged
    sp, sr, sl = C.clone_state(t), C.clone_state(t), C.clone_state(t)
    Pl.step(sp)
    R.step(sr)
    P.step_learned(R, Pl, cn, en, sl, float("inf"))
    er, el = C.field_errors(sr, sp), C.field_errors(sl, sp)
    del sp, sr, sl
    fallbacks, norms = [0], []

    def one():
        fb, r = P.step_learned(R, Pl, cn, en, t, L["max_norm"])
        fallbacks[0] += int(fb)
        norms.append(r)
    ms, clocks = timed_steps(one, nsteps, dev, world, stream, "learned")
    fallbacks_timed = fallbacks[0]
    with P.Profile() as prof:
        one()
    done = args.warmup + nsteps + 1
    for _ in range(max(0, total_steps - done)):
        one()
    finite, ps, t850 = final_diagnostics(P, Pl, t, G.n_cells, dev)
    area = G.cell_areas()
    steps_run = max(total_steps, done)
    out = {"value": job_throughput(world, nsteps, ms), "ms_per_step": ms / nsteps,
           "fallbacks_timed": fallbacks_timed, "fallbacks_warmup": fallbacks_warm,
           "fallbacks_all_steps": fallbacks_warm + fallbacks[0], "steps_run": steps_run,
           "max_norm": L["max_norm"], "check_norm_mean": float(np.nanmean(norms)) if norms else None,
           "finite": finite,
           "rms_ps_pa_vs_fp64": rms_area(area, ps - f64_final["ps"]) if f64_final else None,
           "rms_t850_k_vs_fp64": rms_area(area, t850 - f64_final["t850"]) if f64_final else None,
           "compared_after_steps": steps_run,
           "error_vs_plain_step": {"reduced": er, "learned": el, "ratio": {k: el[k] / er[k] for k in er}},
           "train": {"seconds": train_s, "loss_col": [float(np.mean(lc[:10])), float(np.mean(lc[-50:]))],
                     "loss_edge": [float(np.mean(le[:10])), float(np.mean(le[-50:]))], **{
                         k: (list(v) if isinstance(v, tuple) else v) for k, v in L.items()}},
           "kernels": kernel_table(prof.kernels, 1), "clocks": clocks,
           "hbm_measured": dram_measured("learned", prof.kernels, 1, ms / nsteps,
                                         (G.n_cells, G.n_edges, G.n_verts), nlev, L["ndyn_reduced"])}
    for x in (cn, en, R, Pl):
        x.close()
    del t
    return out


def mixed_summary(m, f64, world, nsteps, area, sizes, nlev, ndyn, leg):
    return {"value": job_throughput(world, nsteps, m["ms"]), "ms_per_step": m["ms"] / nsteps,
            "speedup_vs_fp64": f64["ms"] / m["ms"] if f64 else None, "finite": m["finite"],
            "rms_ps_pa": rms_area(area, m["ps"] - f64["ps"]) if f64 else None,
            "rms_t850_k": rms_area(area, m["t850"] - f64["t850"]) if f64 else None,
            "compared_after_steps": m["steps_run"],
            "reference": "FP64 GPU dycore after the same steps (equal to the FP64 oracle to 1e-12 / 1e-9 after "
                         "1 / 10 steps, GPU parity tests)",
            "hbm_measured": dram_measured(leg, m["prof"], m["nsteps_prof"], m["ms"] / nsteps, sizes, nlev, ndyn),
            "kernels": kernel_table(m["prof"], m["nsteps_prof"]), "clocks": m["clocks"],
            "autotuned_launch_config": m["launch_config"]}


def mountain_legs(P, args, dev, world):
    """The R2B7 L90 Gaussian-mountain configuration (dt 180 s): FP64, mixed and
    mixed + learned over terrain-following heights, timed steps each, the
    mixed legs' surface pressure compared with the FP64 leg's after the same
    number of steps."""
    import numpy as np
    from icon_inputs import make_grid, make_vct, jw_type_state, mountain_height, terrain_following_z
    w = MOUNTAIN
    grid = make_grid(w["bisections"])
    z = make_vct(w["nlev"])
    zz = terrain_following_z(z, mountain_height(grid.cell_xyz, h0=w["h0"], d=w["d"]))
    st0 = jw_type_state(grid, zz, seed=w["seed"])
    G = P.Grid(grid)
    nc, nlev = grid.n_cells, w["nlev"]
    k = min(args.steps, w["max_steps"])
    total = args.warmup + k + 2
    # the exner history starts from the per-column reference state of these heights
    refs = {}

    def prepare(D, st):
        refs["exner"] = D.reference_columns()[1]
        st["exner_pr"] = st["exner"] - refs["exner"]
    area = G.cell_areas()
    sizes = (nc, grid.n_edges, grid.n_verts)
    f64 = measure(P, G, zz, st0, "fp64", args, dev, world, total, w, k, prof_steps=2, prepare=prepare)
    ex_ref = refs["exner"]
    out = {"config": {"workload": "R2B%d L%d (%d cells), Gaussian mountain %.0f m high, %.0f km e-folding radius "
                                  "at 90E 30N, terrain-following heights, dt=%gs, %d substeps + diffusion, JW-type "
                                  "jet seed %d" % (w["bisections"], nlev, nc, w["h0"], w["d"] / 1e3, w["dtime"],
                                                   w["ndyn"], w["seed"]),
                      "steps_timed": k, "max_ground_m": float(zz[:, -1].max())},
           "fp64": {"value": job_throughput(world, k, f64["ms"]), "ms_per_step": f64["ms"] / k,
                    "sdpd": job_throughput(world, k, f64["ms"]) / world * w["dtime"], "finite": f64["finite"],
                    "kernels": kernel_table(f64["prof"], f64["nsteps_prof"]), "clocks": f64["clocks"]}}
    m = measure(P, G, zz, st0, "mixed", args, dev, world, total, w, k, prof_steps=2)
    out["mixed"] = mixed_summary(m, f64, world, k, area, sizes, nlev, w["ndyn"], "mixed")
    out["mixed"]["sdpd"] = out["mixed"]["value"] / world * w["dtime"]
    lrn = learned_leg(P, G, zz, grid, st0, args, dev, world, f64, w, total, k, ex_ref)
    lrn["speedup_vs_fp64"] = lrn["value"] / out["fp64"]["value"]
    lrn["speedup_vs_mixed"] = lrn["value"] / out["mixed"]["value"]
    lrn["sdpd"] = lrn["value"] / world * w["dtime"]
    out["mixed_learned"] = lrn
    G.close()
    return out


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    init_ranks(world, "nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2608_21150_gb300.build import build
    build()
    import paper_2608_21150_gb300 as P
    from icon_inputs import make_grid, make_vct, jw_type_state

    w = WORKLOAD
    grid = make_grid(w["bisections"])
    z = make_vct(w["nlev"])
    nlev = w["nlev"]
    nc, ne, nv = grid.n_cells, grid.n_edges, grid.n_verts
    sizes = (nc, ne, nv)
    st0 = jw_type_state(grid, z, seed=w["seed"])
    G = P.Grid(grid)
    Dref = P.Dycore(G, z, dict(dtime=w["dtime"], ndyn_substeps=w["ndyn"], autotune=0))
    th_ref, ex_ref = Dref.reference_state()
    Dref.close()
    st0["exner_pr"] = st0["exner"] - ex_ref[None, :]
    area = G.cell_areas()
    # every leg runs the same number of steps in all: one simulated day, or at
    # least its warm-up, timed and profiled steps
    day = int(round(86400.0 / w["dtime"])) if args.day else 0
    total = max(day, args.warmup + args.steps + 3)

    legs = set(args.legs.split(","))
    f64, value, ms_per_step, roof, kernels, launches_per_step = None, None, None, None, None, 0
    if "fp64" in legs:
        f64 = measure(P, G, z, st0, "fp64", args, dev, world, total, w, args.steps)
        ms_per_step = f64["ms"] / args.steps
        value = job_throughput(world, args.steps, f64["ms"])
        prof, nsp = f64["prof"], f64["nsteps_prof"]
        launches_per_step = sum(n for n, _ in prof.values()) // nsp
        kernels = kernel_table(prof, nsp)
        roof = roofline(prof, nc, ne, nv, nlev)

    mixed = {}
    for leg in ("mixed", "mixed_f64col"):
        if leg in legs:
            m = measure(P, G, z, st0, leg, args, dev, world, total, w, args.steps)
            mixed[leg] = mixed_summary(m, f64, world, args.steps, area, sizes, nlev, w["ndyn"],
                                       "mixed" if leg == "mixed" else leg)
            mixed[leg]["sdpd"] = mixed[leg]["value"] / world * w["dtime"]

    lrn = None
    if "learned" in legs:
        lrn = learned_leg(P, G, z, grid, st0, args, dev, world, f64, w, total, args.steps, ex_ref[None, :])
        lrn["speedup_vs_fp64"] = lrn["value"] / value if value else None
        lrn["sdpd"] = lrn["value"] / world * w["dtime"]
        if "mixed" in mixed:
            lrn["speedup_vs_mixed"] = lrn["value"] / mixed["mixed"]["value"]

    # end to end through the C-ABI with host arrays (copies inside the timed region)
    sb = state_bytes(nc, ne, nlev)
    e2e = None
    if "fp64" in legs:
        stream = torch.cuda.current_stream(dev)
        e2e_steps = max(5, min(args.steps, 10))
        host = {k: torch.from_numpy(v.copy()).pin_memory() for k, v in st0.items()}
        D2 = P.Dycore(G, z, dict(dtime=w["dtime"], ndyn_substeps=w["ndyn"], rayleigh_coeff=w["rayleigh"],
                                 use_graph=1, synchronous=1, stream=stream.cuda_stream))
        D2.step(host)  # warm-up: allocates the device staging copy and captures the graph
        torch.cuda.synchronize(dev)
        # each call is synchronous (copies in, step, copies out): timed one by
        # one, with Python's garbage collector held off (its pauses are the
        # harness's, not the library's)
        times = []
        gc.disable()
        try:
            for _ in range(e2e_steps):
                t0 = time.perf_counter()
                D2.step(host)
                times.append(time.perf_counter() - t0)
        finally:
            gc.enable()
        D2.close()
        med = statistics.median(times)
        e2e = {"value": 1.0 / med, "unit": "steps/s", "h2d_bytes_per_step": sb, "d2h_bytes_per_step": sb,
               "mean_value": len(times) / sum(times), "step_ms": [round(1e3 * x, 2) for x in times],
               "note": "value at the median wall time of %d synchronous host-array steps (pinned host arrays, "
                       "copies in and out inside each step); mean_value over all of them" % len(times)}
    G.close()
    torch.cuda.empty_cache()

    mountain = mountain_legs(P, args, dev, world) if args.mountain else None

    hbm_bytes = compulsory_bytes_per_step(nc, ne, nlev, w["ndyn"])
    stage_fp64 = stage_bytes_per_step("fp64", nc, ne, nv, nlev, w["ndyn"])
    peak, peak_src = hbm_peak()
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_dict("fp64"),
        "sdpd": value / world * w["dtime"] if value else None,
        "hbm": {"compulsory_bytes_per_step": hbm_bytes,
                "achieved_gbs": hbm_bytes / (ms_per_step / 1000.0) / 1e9,
                "peak_gbs": peak, "peak_source": peak_src,
                "frac": hbm_bytes / (ms_per_step / 1000.0) / 1e9 / peak,
                "stage_bytes_per_step": stage_fp64,
                "stage_frac": stage_fp64 / (ms_per_step / 1000.0) / 1e9 / peak,
                "note": "compulsory (state read+write per substep and diffusion) bytes / step time; "
                        "stage = each field every kernel reads or writes, once per launch; of %s peak" % peak_src}
        if ms_per_step else None,
        "hbm_measured": dram_measured("fp64", f64["prof"], f64["nsteps_prof"], ms_per_step, sizes, nlev, w["ndyn"])
        if f64 else None,
        "roofline": roof,
        "kernels": kernels,
        "autotuned_launch_config": f64["launch_config"] if f64 else None,
        "steps_compared": total,
        "mixed": mixed.get("mixed"),
        "mixed_f64col": mixed.get("mixed_f64col"),
        "mixed_learned": lrn,
        "mountain_r2b7": mountain,
        "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": f64["clocks"] if f64 else None, "finite": f64["finite"] if f64 else None,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(nlev)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--legs", default="fp64,mixed,mixed_f64col,learned",
                    help="comma-separated legs to run (fp64, mixed, mixed_f64col, learned); the headline value is "
                         "the fp64 leg's")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision and learned legs")
    ap.add_argument("--no-learned", action="store_true", help="skip the mixed + learned-corrector leg")
    ap.add_argument("--no-day", dest="day", action="store_false",
                    help="compare the legs after their own steps instead of one simulated day")
    ap.add_argument("--no-mountain", dest="mountain", action="store_false",
                    help="skip the R2B7 Gaussian-mountain section")
    ap.add_argument("--grid", type=int, default=WORKLOAD["bisections"],
                    help="RnBm bisections (default 6 = R2B6); other grids for profiler captures and scaling runs")
    ap.add_argument("--dtime", type=float, default=WORKLOAD["dtime"],
                    help="time step in s (default 360, the R2B6 step; 180 at R2B7)")
    ap.add_argument("--fused-advection", action="store_true",
                    help="mixed legs: the velocity tendencies in the one fused kernel over cell patches "
                         "instead of four kernels (same bits, slower on GB300)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    WORKLOAD["bisections"] = args.grid
    WORKLOAD["dtime"] = args.dtime
    WORKLOAD["fused_advection"] = int(args.fused_advection)
    legs = [x for x in args.legs.split(",") if x]
    if args.no_mixed:
        legs = [x for x in legs if x not in ("mixed", "mixed_f64col", "learned")]
    if args.no_learned:
        legs = [x for x in legs if x != "learned"]
    if any(x not in ("fp64", "mixed", "mixed_f64col", "learned") for x in legs):
        ap.error("--legs takes fp64, mixed, mixed_f64col, learned")
    args.legs = ",".join(legs)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
