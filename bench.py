#!/usr/bin/env python
"""Throughput of the GB300 ICON-type dycore step on R2B6 L90.

Workload (the configuration the headline metric is quoted on): icosahedral
R2B6 grid (327 680 cells, 491 520 edges), 90 levels to 30 km, dt = 360 s,
5 dynamical substeps + diffusion per step, Rayleigh damping above 20 km,
balanced JW-type baroclinic jet with the seeded Gaussian perturbation
(seed 2).  Synthetic inputs (no dataset exists in this environment).

A "step" is one full dycore time step.  The device-resident leg times K
steps replayed as one CUDA graph each, with CUDA events on the stream the
library launches on; the state (1.5 GB) is larger than L2, so no flush is
needed.  The end-to-end leg calls the C-ABI with HOST arrays: the library
copies the state in and out around every step.  The mixed leg runs the same
steps with FP32 stencils; the mixed + learned leg trains the corrector on the
GPU (untimed, other seeds), then times steps with 4 substeps plus the learned
increments, the check and any fallback to the plain step.  N>1 (torchrun) runs N
independent replicas (ensemble members), one per GPU.

``--impl reference`` times the FP64 CPU oracle instead (on the host cores),
each step a bounded sample: one substep and one diffusion call on R2B4 L90,
scaled to a full R2B6 L90 step (x5 substeps, x16 cells).
"""
import argparse
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
SAMPLE_BISECTIONS = 4          # reference / cpu_baseline sample grid (1/16 of the R2B6 columns)
METRIC = "dycore steps/s + HBM GB/s fraction at R2B6 L90: FP64 vs mixed+learned"
FP64_PEAK_TFLOPS = 1.25        # nominal GB300 FP64 (152 SMs x 2 DFMA/clk x 2 flop x ~2.06 GHz)

# Algorithmic FP64 flops per unit (FMA = 2, add/mul/div/sqrt = 1), counted
# from the formulas each kernel evaluates; the unit is one (point, level).
FLOPS_PER_UNIT = {
    "va_edge_pre": 13, "va_cell_vert": 17, "va_edge_tend": 38, "va_cell_w": 13,
    "sn_cell_grad": 28, "sn_edge_pred": 38, "sn_cell_div": 5, "sn_cell_fluxdiv": 27,
    "sn_column_pred": 86, "sn_edge_corr": 17, "sn_column_corr": 94,
    "diff_div_curl_uv": 30, "diff_edge_smag": 46, "diff_second": 30,
    "diff_edge_update": 12, "diff_cell_update": 12,
}


def units_per_launch(name, nc, ne, nv, nlev):
    full = {"c": nc * nlev, "e": ne * nlev, "v": nv * nlev}
    half = {"c": nc * (nlev + 1), "e": ne * (nlev + 1), "v": nv * (nlev + 1)}
    return {
        "va_edge_pre": full["e"], "va_cell_vert": full["c"] + half["v"], "va_edge_tend": half["e"],
        "va_cell_w": half["c"], "sn_cell_grad": full["c"], "sn_edge_pred": full["e"],
        "sn_column_pred": full["c"], "sn_edge_corr": full["e"], "sn_column_corr": full["c"],
        "sn_cell_div": full["c"], "sn_cell_fluxdiv": full["c"],
        "diff_div_curl_uv": full["c"] + full["v"], "diff_edge_smag": full["e"],
        "diff_second": half["c"] + full["v"], "diff_edge_update": full["e"], "diff_cell_update": half["c"],
    }[name]


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


def oracle_sample(bisections, nlev, reps):
    """Time the oracle (as it stands) on one substep and one diffusion call of
    the given grid, in a fresh single-threaded process; returns seconds."""
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
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if p.returncode != 0:
        raise RuntimeError(p.stderr)
    return json.loads(p.stdout.strip().splitlines()[-1])


def sample_to_steps_per_s(t_sub, t_diff, scale):
    return 1.0 / (scale * (WORKLOAD["ndyn"] * t_sub + t_diff))


def cpu_baseline(nlev):
    samples = oracle_sample(SAMPLE_BISECTIONS, nlev, 1)
    t_sub, t_diff = samples[0]
    scale = 4 ** (WORKLOAD["bisections"] - SAMPLE_BISECTIONS)
    return {"value": sample_to_steps_per_s(t_sub, t_diff, scale), "unit": "steps/s", "cores": 1,
            "kind": "oracle",
            "sample": "one substep (%.1f s) + one diffusion (%.1f s) of the numpy FP64 oracle on R2B4 L90 "
                      "(1/16 of the R2B6 columns), scaled to an R2B6 L90 step as 16 x (5 substeps + diffusion)"
                      % (t_sub, t_diff)}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    nlev = WORKLOAD["nlev"]
    reps = args.warmup + args.steps
    samples = oracle_sample(SAMPLE_BISECTIONS, nlev, reps)[args.warmup:]
    scale = 4 ** (WORKLOAD["bisections"] - SAMPLE_BISECTIONS)
    step_s = [scale * (WORKLOAD["ndyn"] * a + b) for a, b in samples]
    total = sum(step_s)
    value = args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_dict("fp64"),
        "cpu_baseline": {"value": value, "unit": "steps/s", "cores": 1, "kind": "oracle",
                         "sample": "per step: one substep + one diffusion of the numpy FP64 oracle on R2B4 L90, "
                                   "scaled x16 (cells) and x5 (substeps) to an R2B6 L90 step"},
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


def measure(P, G, z, st0, prec, args, dev, world):
    """Time K steps of one precision mode; returns the numbers and the final state."""
    import torch
    import torch.distributed as dist
    w = WORKLOAD
    stream = torch.cuda.current_stream(dev)
    D = P.Dycore(G, z, dict(dtime=w["dtime"], ndyn_substeps=w["ndyn"], rayleigh_coeff=w["rayleigh"],
                            precision=P.ICON_PREC_MIXED if prec == "mixed" else P.ICON_PREC_FP64,
                            use_graph=1, synchronous=0, stream=stream.cuda_stream))
    t = {k: torch.from_numpy(v).to(dev) for k, v in st0.items()}
    for _ in range(args.warmup):
        D.step(t)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(dev.index)
    sampler.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    torch.cuda.nvtx.range_push(prec + "_timed")   # marks the timed steps for profiler filters
    e0.record(stream)
    for _ in range(args.steps):
        D.step(t)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    if world > 1:
        dist.barrier()
    ms = max_over_ranks(ms, world, dev)
    nc = G.n_cells
    ps = torch.empty(nc, dtype=torch.float64, device=dev)
    t850 = torch.empty_like(ps)
    try:
        D.diagnostics(t, ps, t850)
        finite = True
    except P.IconError:
        finite = False
    out = dict(ms=ms, clocks=clocks, finite=finite, ps=ps.cpu().numpy(), t850=t850.cpu().numpy())
    nsteps_prof = min(args.steps, 3)
    out["prof"] = D.profile(t, nsteps_prof)
    out["nsteps_prof"] = nsteps_prof
    out["launch_config"] = D.launch_config()
    D.close()
    return out, t


LEARNED = dict(ndyn_reduced=4, hidden=512, max_batch=65536, train_seeds=(100, 101, 102, 103), spinup=1,
               snapshots=8, every=3, rows=8192, adam_steps=1500, batch=4096, lr=1e-3, max_norm=3.0)


def learned_leg(P, G, z, grid, st0, args, dev, world, f64_final):
    """Mixed precision + learned corrector: a step with ndyn_reduced substeps,
    the column and edge networks' increments, the norm/finiteness check and the
    plain-step fallback (icon_dycore_step_learned).  The corrector is trained
    first on the GPU (untimed) from paired reduced/plain steps of other seeds."""
    import numpy as np
    import torch
    from paper_2608_21150_gb300 import corrector as C
    w, L = WORKLOAD, LEARNED
    stream = torch.cuda.current_stream(dev)
    base = dict(dtime=w["dtime"], rayleigh_coeff=w["rayleigh"], precision=P.ICON_PREC_MIXED, use_graph=1,
                synchronous=0, stream=stream.cuda_stream)
    R = P.Dycore(G, z, dict(base, ndyn_substeps=L["ndyn_reduced"]))
    Pl = P.Dycore(G, z, dict(base, ndyn_substeps=w["ndyn"]))
    ex_ref = R.reference_state()[1]
    t0 = time.perf_counter()
    gen = torch.Generator()
    gen.manual_seed(0)
    data = C.Dataset()
    from icon_inputs import jw_type_state
    for seed in L["train_seeds"]:
        s0 = jw_type_state(grid, z, seed=seed)
        s0["exner_pr"] = s0["exner"] - ex_ref[None, :]
        st = {k: torch.from_numpy(v).to(dev) for k, v in s0.items()}
        for _ in range(L["spinup"]):
            Pl.step(st)
        for _ in range(L["snapshots"]):
            st = C.add_pair(R, Pl, st, data, rows=L["rows"], gen=gen)
            for _ in range(L["every"] - 1):
                Pl.step(st)
    cx, cy, ex, ey = data.cat()
    del data
    cn, en = C.make_nets(w["nlev"], hidden=L["hidden"], max_batch=L["max_batch"], seed=1)
    lc = C.fit(cn, cx, cy, w["nlev"], L["adam_steps"], batch=L["batch"], lr=L["lr"])
    le = C.fit(en, ex, ey, w["nlev"], L["adam_steps"], batch=L["batch"], lr=L["lr"])
    del cx, cy, ex, ey
    torch.cuda.synchronize(dev)
    train_s = time.perf_counter() - t0

    t = {k: torch.from_numpy(v).to(dev) for k, v in st0.items()}
    fallbacks_warm = 0
    for _ in range(args.warmup):
        fb, _ = P.step_learned(R, Pl, cn, en, t, L["max_norm"])
        fallbacks_warm += int(fb)
    # held-out error of the corrector at the bench state (reduced and learned vs the plain step)
    sp, sr, sl = C.clone_state(t), C.clone_state(t), C.clone_state(t)
    Pl.step(sp)
    R.step(sr)
    P.step_learned(R, Pl, cn, en, sl, float("inf"))
    er, el = C.field_errors(sr, sp), C.field_errors(sl, sp)
    del sp, sr, sl
    torch.cuda.synchronize(dev)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    sampler = ClockSampler(dev.index)
    sampler.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    fallbacks, norms = 0, []
    torch.cuda.nvtx.range_push("learned_timed")
    e0.record(stream)
    for _ in range(args.steps):
        fb, r = P.step_learned(R, Pl, cn, en, t, L["max_norm"])
        fallbacks += int(fb)
        norms.append(r)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    nc = G.n_cells
    ps = torch.empty(nc, dtype=torch.float64, device=dev)
    t850 = torch.empty_like(ps)
    try:
        Pl.diagnostics(t, ps, t850)
        finite = True
    except P.IconError:
        finite = False
    area = G.cell_areas()
    rms = lambda d: float(np.sqrt(np.sum(area * d ** 2) / np.sum(area)))  # noqa: E731
    with P.Profile() as prof:
        P.step_learned(R, Pl, cn, en, t, L["max_norm"])
    out = {"value": job_throughput(world, args.steps, ms), "ms_per_step": ms / args.steps,
           "fallbacks_timed": fallbacks, "fallbacks_warmup": fallbacks_warm, "max_norm": L["max_norm"],
           "check_norm_mean": float(np.nanmean(norms)) if norms else None, "finite": finite,
           "rms_ps_pa_vs_fp64": rms(ps.cpu().numpy() - f64_final["ps"]) if f64_final else None,
           "rms_t850_k_vs_fp64": rms(t850.cpu().numpy() - f64_final["t850"]) if f64_final else None,
           "error_vs_plain_step": {"reduced": er, "learned": el,
                                   "ratio": {k: el[k] / er[k] for k in er}},
           "train": {"seconds": train_s, "loss_col": [float(np.mean(lc[:10])), float(np.mean(lc[-50:]))],
                     "loss_edge": [float(np.mean(le[:10])), float(np.mean(le[-50:]))], **{
                         k: (list(v) if isinstance(v, tuple) else v) for k, v in L.items()}},
           "hbm_measured": dram_measured("learned", ms / args.steps),
           "kernels": kernel_table(prof.kernels, 1), "clocks": clocks}
    for x in (cn, en, R, Pl):
        x.close()
    return out


# The column solve's predictor and corrector launches are one kernel (one
# function, two forms); the roofline treats them together.
FAMILY = {"sn_column_pred": "sn_column", "sn_column_corr": "sn_column"}

# DRAM bytes per launch of the FP64 column solve (the mean of its predictor
# and corrector launches, 6.39 and 8.47 GB) from the ncu capture of the FP64
# step at R2B6 L90, valid for that grid
# while the kernel source is the one captured (its SHA-256 below).
COLUMN_TRAFFIC = {"source": "paper_2608_21150_gb300/csrc/kernels_column.cu",
                  "sha256": "1fc4e7a652e5d510c7db7dfe44654c9b8fd3a81b01462c4eac418754c02a58ea",
                  "bisections": 6, "bytes_per_launch": 7.427e9}


# DRAM bytes per step of every kernel in the timed steps, from one ncu capture
# of each leg at R2B6 L90, valid while
# the kernel sources are the ones captured (SHA-256 over csrc/* except the
# host-only set-up code, below).
STEP_DRAM = {"sources_sha256": "987083fa96c2d1d9b02eead4bb1f78ece04babebba2a12334617df53cb029a45",
             "bisections": 6, "bytes_per_step": {"fp64": 207.265e9, "mixed": 154.345e9,
                                                 "learned": 134.728e9}}


# Host-only set-up code (grid validation and geometry factors, run untimed at
# create) cannot change a kernel's DRAM traffic and is left out of the hash.
HOST_ONLY_SOURCES = ("grid_setup.cpp",)


def sources_sha256():
    """sha256 over the library sources that shape the timed kernels' traffic."""
    import glob
    import hashlib
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_2608_21150_gb300", "csrc", "*"))):
        if os.path.basename(f) in HOST_ONLY_SOURCES:
            continue
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def dram_measured(leg, ms_per_step):
    """Measured DRAM bytes per step (ncu) over the live step time: achieved HBM
    GB/s and its fraction of the measured peak, and the traffic amplification
    (measured over algorithmic stage bytes); null if the kernels changed since
    the capture or the grid is not the captured one."""
    t = STEP_DRAM
    if WORKLOAD["bisections"] != t["bisections"] or sources_sha256() != t["sources_sha256"]:
        return None
    b = t["bytes_per_step"][leg]
    gbs = b / (ms_per_step / 1000.0) / 1e9
    nc = 80 * 4 ** WORKLOAD["bisections"]
    stage = stage_bytes_per_step(leg, nc, 3 * nc // 2, nc // 2 + 2, WORKLOAD["nlev"], WORKLOAD["ndyn"])
    return {"bytes_per_step": b, "achieved_gbs": gbs, "peak_gbs": 6663.9, "frac": gbs / 6663.9,
            "stage_bytes_per_step": stage, "amplification": b / stage if stage else None,
            "note": "ncu dram__bytes_read.sum + dram__bytes_write.sum over all kernels of the timed steps / "
                    "event-timed step; of measured peak; amplification = these bytes / the algorithmic stage "
                    "bytes (each field a kernel reads or writes, once per launch)"}


def column_traffic():
    import hashlib
    t = COLUMN_TRAFFIC
    if WORKLOAD["bisections"] != t["bisections"]:
        return None
    try:
        with open(os.path.join(ROOT, t["source"]), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != t["sha256"]:
                return None
    except OSError:
        return None
    return t["bytes_per_launch"]


def roofline(prof, nc, ne, nv, nlev):
    """FP64-ALU roofline of the kernel family with the largest share of the step."""
    fam = {}
    for k, (n, ms) in prof.items():
        f = FAMILY.get(k, k)
        flops = FLOPS_PER_UNIT[k] * units_per_launch(k, nc, ne, nv, nlev) * n
        a = fam.setdefault(f, [0, 0.0, 0.0])
        a[0] += n
        a[1] += ms
        a[2] += flops
    name, (n, ms, flops) = max(fam.items(), key=lambda kv: kv[1][1])
    achieved = flops / (ms / 1000.0) / 1e12
    return {"bound": "alu", "kernel": name, "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS,
            "traffic": column_traffic() if name == "sn_column" else None,
            "note": "FP64 algorithmic flops per launch / event-timed launch duration (CUDA events around every "
                    "launch on the library's stream); peak = nominal FP64 rate from unit counts and clock "
                    "(1.2 TFLOP/s measured by a DFMA probe); traffic = ncu DRAM bytes per launch"}


def kernel_table(prof, nsteps):
    tot = sum(v[1] for v in prof.values()) / nsteps
    return {k: {"launches_per_step": n // nsteps, "ms_per_step": round(m / nsteps, 3),
                "share": round(m / nsteps / tot, 4)} for k, (n, m) in sorted(prof.items(), key=lambda kv: -kv[1][1])}


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
    st0 = jw_type_state(grid, z, seed=w["seed"])
    G = P.Grid(grid)
    Dref = P.Dycore(G, z, dict(dtime=w["dtime"], ndyn_substeps=w["ndyn"]))
    th_ref, ex_ref = Dref.reference_state()
    Dref.close()
    st0["exner_pr"] = st0["exner"] - ex_ref[None, :]

    legs = set(args.legs.split(","))
    f64, value, ms_per_step, roof, kernels, launches_per_step = None, None, None, None, None, 0
    if "fp64" in legs:
        f64, _ = measure(P, G, z, st0, "fp64", args, dev, world)
        ms_per_step = f64["ms"] / args.steps
        value = job_throughput(world, args.steps, f64["ms"])
        prof, nsp = f64["prof"], f64["nsteps_prof"]
        launches_per_step = sum(n for n, _ in prof.values()) // nsp
        kernels = kernel_table(prof, nsp)
        roof = roofline(prof, nc, ne, nv, nlev)

    mx = None
    if "mixed" in legs:
        m, _ = measure(P, G, z, st0, "mixed", args, dev, world)
        area = G.cell_areas()
        rms = lambda d: float(np.sqrt(np.sum(area * d ** 2) / np.sum(area)))  # noqa: E731
        mx = {"value": job_throughput(world, args.steps, m["ms"]), "ms_per_step": m["ms"] / args.steps,
              "speedup_vs_fp64": f64["ms"] / m["ms"] if f64 else None, "finite": m["finite"],
              "rms_ps_pa": rms(m["ps"] - f64["ps"]) if f64 else None,
              "rms_t850_k": rms(m["t850"] - f64["t850"]) if f64 else None,
              "compared_after_steps": args.warmup + args.steps,
              "reference": "FP64 GPU dycore (equal to the FP64 oracle to 1e-9 after 10 steps, GPU parity tests)",
              "hbm_measured": dram_measured("mixed", m["ms"] / args.steps),
              "kernels": kernel_table(m["prof"], m["nsteps_prof"]), "clocks": m["clocks"],
              "autotuned_launch_config": m["launch_config"]}

    lrn = None
    if "learned" in legs:
        lrn = learned_leg(P, G, z, grid, st0, args, dev, world, f64)
        lrn["speedup_vs_fp64"] = lrn["value"] / value if value else None
        if mx:
            lrn["speedup_vs_mixed"] = lrn["value"] / mx["value"]

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
        # each call is synchronous (copies in, step, copies out): timed one by one
        times = []
        for _ in range(e2e_steps):
            t0 = time.perf_counter()
            D2.step(host)
            times.append(time.perf_counter() - t0)
        D2.close()
        med = statistics.median(times)
        e2e = {"value": 1.0 / med, "unit": "steps/s", "h2d_bytes_per_step": sb, "d2h_bytes_per_step": sb,
               "mean_value": len(times) / sum(times), "step_ms": [round(1e3 * x, 2) for x in times],
               "note": "value at the median wall time of %d synchronous host-array steps (pinned host arrays, "
                       "copies in and out inside each step); mean_value over all of them" % len(times)}

    hbm_bytes = compulsory_bytes_per_step(nc, ne, nlev, w["ndyn"])
    stage_fp64 = stage_bytes_per_step("fp64", nc, ne, nv, nlev, w["ndyn"])
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_dict("fp64"),
        "sdpd": value / world * w["dtime"] if value else None,
        "hbm": {"compulsory_bytes_per_step": hbm_bytes,
                "achieved_gbs": hbm_bytes / (ms_per_step / 1000.0) / 1e9,
                "peak_gbs": 6663.9, "frac": hbm_bytes / (ms_per_step / 1000.0) / 1e9 / 6663.9,
                "stage_bytes_per_step": stage_fp64,
                "stage_frac": stage_fp64 / (ms_per_step / 1000.0) / 1e9 / 6663.9,
                "note": "compulsory (state read+write per substep and diffusion) bytes / step time; "
                        "stage = each field every kernel reads or writes, once per launch; of measured peak"}
        if ms_per_step else None,
        "hbm_measured": dram_measured("fp64", ms_per_step) if ms_per_step else None,
        "roofline": roof,
        "kernels": kernels,
        "autotuned_launch_config": f64["launch_config"] if f64 else None,
        "mixed": mx,
        "mixed_learned": lrn,
        "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": f64["clocks"] if f64 else None, "finite": f64["finite"] if f64 else None,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(nlev)
    if rank == 0:
        print(json.dumps(line))
    G.close()
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
    ap.add_argument("--legs", default="fp64,mixed,learned",
                    help="comma-separated legs to run (fp64, mixed, learned); the headline value is the fp64 leg's")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision and learned legs")
    ap.add_argument("--no-learned", action="store_true", help="skip the mixed + learned-corrector leg")
    ap.add_argument("--grid", type=int, default=WORKLOAD["bisections"],
                    help="RnBm bisections (default 6 = R2B6); other grids for profiler captures and scaling runs")
    ap.add_argument("--dtime", type=float, default=WORKLOAD["dtime"],
                    help="time step in s (default 360, the R2B6 step; 180 at R2B7)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    WORKLOAD["bisections"] = args.grid
    WORKLOAD["dtime"] = args.dtime
    legs = [x for x in args.legs.split(",") if x]
    if args.no_mixed:
        legs = [x for x in legs if x not in ("mixed", "learned")]
    if args.no_learned:
        legs = [x for x in legs if x != "learned"]
    if any(x not in ("fp64", "mixed", "learned") for x in legs):
        ap.error("--legs takes fp64, mixed, learned")
    args.legs = ",".join(legs)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
