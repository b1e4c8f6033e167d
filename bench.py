"""Throughput benchmark of the fused, batched PWF iteration on GB300.

Workload (default): a tomographic series of 180 projections of 1024 x 1024
pixels (angles 0..179 degrees of a seeded 40-ellipsoid phantom, 20 keV, 1 um
pixels, L1 = 0.1 m, L2 = 0.4 m), shared diffuser, partial coherence in the
paper's IOTF form (Gaussian blur of sigma = 2 px), gamma = 1, alpha = 0.1 +
0.01i. One step = one PWF iteration (Algorithm S1 body: forward model,
residual, Wirtinger derivative, preconditioner + regularizer, Nesterov) over
all 180 projections. Metric: megapixel-projection iterations per second.

Arms:
  default            fused batched CUDA path (libpwf, pwf_solve), plus the
                     unfused per-projection baseline (PWF_FLAG_PLAIN) on a
                     sample, the roofline of the dominant kernel, the FP64
                     oracle on the host cores (cpu_baseline) and an
                     end-to-end number through host buffers (pwf_solve_host:
                     pinned y and t in, psi out, copies overlapping the
                     solve; every rank, max over ranks).
  --impl reference   the FP64 oracle on the host cores, timed per step on a
                     bounded sample of the same workload.

Multi-GPU (torchrun): every rank runs its own 180-projection series (weak
scaling, no collective on the data path); the timed region is bracketed by a
barrier and the max over ranks is reported.
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

METRIC = "megapixel-projection PWF iterations/s at 1 GB300 (fused batched vs plain); % HBM roofline"
UNIT = "Mpx*it/s"

# Algorithmic DRAM bytes per pixel of each pass of the fused iteration (reads +
# writes of the fields the pass must touch; complex64 = 8 B, float32 = 4 B).
STATE_FLOOR_BYTES_PER_PX = 44  # psi r/w 16, phi r 8 + w 8, t 8, y 4

PASS_BYTES_PER_PX = {
    "col_q": 16,            # field in, field out
    "row_mul_t": 24,        # field in, t in, field out
    "row_intensity": 24,    # field in, v out, F_row{|v|^2} out
    "col_resid_iotf2": 24,  # field in, F{y} in, field out
    "row_mul_v": 24,        # field in, v in, field out
    "row_grad_pack": 36,    # field in, psi in, Re g out, two fields out
    "col_precond_reg": 24,  # two fields in, one out
    "row_nesterov_fft": 52, # field, psi, phi, Re g in; phi, psi, field out
    "row_coh_resid": 20,    # field in, y in, field out
    # packed residual passes (two real rows per complex row; bins 0..nx/2)
    "row_intensity_pk": 20, # field in, v out, packed F_row{|v|^2} out (4 B/px)
    "col_resid_pk": 12,     # packed field in and out (4 + 4), F{y} of bins 0..nx/2 (4)
    "row_mul_v_pk": 20,     # packed field in (4), v in, field out
    # source-mode variant (per mode; see modal_bytes_per_px)
    "col_mode_fwd": 16,     # shifted column in, field out
    "row_mode_int": 24,     # field in, v_j out, intensity accumulated
    "modal_resid": 12,      # intensity, y in; G out
    "row_mode_vg": 20,      # v_j, G in; field out
    "col_mode_back": 24,    # field in, spectrum accumulated
    "col_fft": 16,          # F_row{x} -> 2-D spectrum, in place
    "col_ifft": 16,         # accumulated spectrum -> F_row, in place
    "finalize": 0,
}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tomo180x1024_iotf")
    ap.add_argument("--batch", type=int, default=None, help="override projections per GPU")
    ap.add_argument("--no-extras", action="store_true", help="skip plain/e2e/cpu legs")
    ap.add_argument("--column-shapes", default=None,
                    help="comma list of column-shape indices (one per column op, in pass order) forced after the plan-time "
                         "tuning of the main plan, e.g. the column_shape_ids of an earlier line")
    ap.add_argument("--legs", default="all",
                    help="comma list of extra legs to run (plain,e2e,modal,small,mixed,autograd,fbp,ablation,cpu) "
                         "or all")
    return ap.parse_args()


# ----------------------------------------------------------------------------
# distributed plumbing
# ----------------------------------------------------------------------------
def dist_setup(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples go to PWF_CLOCKS_DIR (default: the system temp directory)
        out = os.environ.get("PWF_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out, f"clocks_rank{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            # nvidia-smi takes a moment to start: let its first sample land
            # before the timed region opens, so that the region is covered
            t0 = time.time()
            while time.time() - t0 < 3.0 and self.proc.poll() is None:
                if os.path.getsize(self.path) > 0:
                    break
                time.sleep(0.02)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                except ValueError:
                    continue
                for name, val in zip(names, f[5:9]):
                    if val.lower() == "active":
                        reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------
# workload synthesis (seeded; on the GPU for speed)
# ----------------------------------------------------------------------------
def make_workload(P, S, w, batch, device, rank=0, world=1):
    """Rank r of `world` takes its cost-balanced share of a world*batch-angle
    series (shard.shard_projections; weak scaling: each rank solves its own
    batch of distinct projections, no exchange during the iterations)."""
    import numpy as np
    import torch
    from paper_2503_20146_gb300 import shard
    n = w.ny
    if w.name.startswith("tomo"):
        ph = S.ellipsoid_phantom(S.rng_for(w.config, 0), size=n)
        xd, yd = S.detector_grid(n, n, xp=torch)
        xd, yd = xd.to(device), yd.to(device)
        angles = S.tomo_angles(batch * world)
        mine = shard.shard_projections([(n, n, w.n_modes)] * (batch * world), world, rank)
        psi_true = torch.empty((len(mine), n, n), dtype=torch.complex64, device=device)
        for i, ang in enumerate(angles[mine]):
            re, im = S.ellipsoid_projection(ph, float(ang), xd, yd, w.wavelength_m)
            psi_true[i] = torch.complex(re, im).to(torch.complex64)
    else:
        psi_true = torch.stack([torch.from_numpy(S.complex_phase_from(
            S.blob_phase(w.ny, w.nx, S.rng_for(w.config, b))).astype(np.complex64)) for b in range(batch)]).to(device)
    t = torch.from_numpy(S.diffuser(w.ny, w.nx, S.rng_for(w.config, 99)).astype(np.complex64)).to(device)
    return psi_true, t


# Algorithmic bytes per pixel of one source-mode iteration (K modes): per mode
# the forward CM_FWD 16, ROW_MUL_T 24, COL_Q 16, ROW_MODE_INT 24 (v_j stored,
# intensity accumulated) and the backward ROW_MODE_VG 20, COL_Q 16, ROW_MUL_T 24,
# CM_BACK 24 (spectrum accumulated) = 164 B/px; once per iteration the residual
# 12 and ROW_GRAD_PACK + COL_PRECOND_REG + ROW_NESTEROV_FFT 112.
def modal_bytes_per_px(k: int) -> int:
    # per mode 164; residual 12; COL_FFT of F_row{x} and COL_IFFT of the
    # accumulated spectrum 16 each; GRAD_PACK, PRECOND_REG, NESTEROV 112
    return 164 * k + 12 + 32 + 112


def plan_desc(P, w, batch, flags=0, n_modes=None):
    return P.PlanDesc(batch, w.ny, w.nx, w.pixel_m, w.wavelength_m, w.L1_m, w.L2_m, w.xcoh_m, w.ycoh_m,
                      w.gamma, w.alpha.real, w.alpha.imag, w.eta, flags,
                      w.n_modes if n_modes is None else n_modes, w.mode_sigma_px)


def selected_shape_ids(describe: str):
    """Index of the chosen shape of every column op in its candidate list, read
    from pwf_plan_describe ("op=NAME[NAME:ms,...]"); None where not tuned."""
    import re
    ids = []
    for m in re.finditer(r" col_[a-z0-9_]+=([^\[ ]+)(?:\[([^\]]*)\])?", describe):
        names = [c.rsplit(":", 1)[0] for c in m.group(2).split(",")] if m.group(2) else []
        ids.append(names.index(m.group(1)) if m.group(1) in names else None)
    return ids


def source_hash():
    """Hash of the files that define the pass kernels (templates and their
    per-length instantiations): stored DRAM counters stay valid while it holds."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2503_20146_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if not (name in ("fft.cuh", "passes.cuh", "pass_types.h") or name.startswith("len_")):
            continue
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(name.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None
    when the summary was taken on other kernel sources."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except Exception:
        return None
    if d.get("source_hash") != source_hash():
        return None
    k = d.get("kernels", {}).get(kernel)
    return None if k is None else k.get("dram_bytes_per_launch_full")


SCHEDULERS_PER_SM = 4  # warp schedulers (SM sub-partitions) per SM, one instruction each per cycle


def issue_roofline(inst_per_px, px, launch_ms, sms, sm_mhz):
    """Warp-instruction issue rate of one launch against the SMs' peak issue
    rate (every scheduler issuing every cycle at sm_mhz)."""
    achieved = inst_per_px * px / 32.0 / (launch_ms / 1e3) / 1e9
    peak = sms * SCHEDULERS_PER_SM * sm_mhz * 1e6 / 1e9
    return {"achieved": achieved, "peak": peak, "unit": "G warp-instructions/s", "frac": achieved / peak,
            "thread_instructions_per_px": inst_per_px, "sm_mhz": sm_mhz}


def measured_instructions_per_px(kernel):
    """Thread instructions per pixel of `kernel` from the committed ncu summary
    (smsp__inst_executed.sum x 32 / captured pixels), or None when the summary
    was taken on other kernel sources."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except Exception:
        return None
    if d.get("source_hash") != source_hash():
        return None
    k = d.get("kernels", {}).get(kernel) or {}
    if "warp_instructions" not in k or "captured_px" not in k:
        return None
    return k["warp_instructions"] * 32.0 / k["captured_px"]


def max_sm_mhz():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["sm_max_mhz"])
    except Exception:
        return None


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------------------------
# oracle timing on the host (cpu_baseline and the reference arm)
# ----------------------------------------------------------------------------
CPU_SAMPLE_ITERS = 12  # ~0.5-1 s per 1024^2 iteration on one host core


def oracle_job(wname, b, iters):
    """The unchanged FP64 oracle on projection b of the workload's size (blob
    measurements stand in for the phantom: the oracle's cost does not depend
    on the values) for `iters` iterations, in a worker process; returns the
    seconds the solve took."""
    import numpy as np
    from oracle import pwf_oracle as O
    from paper_2503_20146_gb300 import synth as S
    w = S.WORKLOADS[wname]
    geom = O.Geometry(w.ny, w.nx, w.pixel_m, w.wavelength_m, w.L1_m, w.L2_m, w.xcoh_m, w.ycoh_m, w.gamma,
                      w.alpha, w.eta)
    t = S.diffuser(w.ny, w.nx, S.rng_for(w.config, 99))
    y = np.clip(1.0 + 0.1 * S.rng_for(w.config, 200 + b).standard_normal((w.ny, w.nx)), 0, None)
    t0 = time.perf_counter()
    O.solve(y, t, geom, iters)
    return time.perf_counter() - t0


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


class OraclePool:
    """One worker process per host core (spawn: the parent already holds a
    CUDA context), each running the oracle single-threaded on its own
    projection; a sample is `cores` projections solved at once."""

    def __init__(self, cores=None):
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        self.cores = cores or host_cores()
        self.ex = ProcessPoolExecutor(max_workers=self.cores, mp_context=mp.get_context("spawn"))

    def sample(self, w, iters):
        """Wall-clock seconds for `cores` projections x `iters` iterations, and the Mpx*it done."""
        t0 = time.perf_counter()
        list(self.ex.map(oracle_job, [w.name] * self.cores, range(self.cores), [iters] * self.cores))
        return time.perf_counter() - t0, self.cores * w.ny * w.nx * iters / 1e6

    def close(self):
        self.ex.shutdown()


def run_reference(args, w, rank, world):
    if rank != 0:
        return
    # one step = one oracle iteration on each of `cores` projections, one
    # worker process per host core
    pool = OraclePool()
    for _ in range(args.warmup):
        pool.sample(w, 1)
    times, work = [], 0.0
    for _ in range(args.steps):
        dt, mpx = pool.sample(w, 1)
        times.append(dt)
        work += mpx
    pool.close()
    total = sum(times)
    value = work / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"{w.name}: oracle on {pool.cores} of {w.batch} projections per step",
                   "ny": w.ny, "nx": w.nx, "batch": w.batch},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
                         "sample": f"{pool.cores} projections of {w.ny}x{w.nx} (one per core, worker "
                                   f"processes), 1 iteration per step, numpy FP64"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_mixed(P, S, torch, dev, stream, steps=4):
    """One group of four size-class plans; seeded blob objects, the CUDA
    forward model and Poisson noise at per-projection photon counts."""
    import numpy as np
    wm = S.WORKLOADS["mixed64_k25"]
    plans, ys, ts, psis = [], [], [], []
    mpx = 0.0
    for ci, n in enumerate(S.MIXED_SIZES):
        d = P.PlanDesc(S.MIXED_PER_SIZE, n, n, wm.pixel_m, wm.wavelength_m, wm.L1_m, wm.L2_m, wm.xcoh_m, wm.ycoh_m,
                       wm.gamma, wm.alpha.real, wm.alpha.imag, wm.eta, 0, wm.n_modes, wm.mode_sigma_px)
        plan = P.Plan(d)
        psi_true = torch.empty((S.MIXED_PER_SIZE, n, n), dtype=torch.complex64, device=dev)
        for b in range(S.MIXED_PER_SIZE):
            phi = S.blob_phase(n, n, S.rng_for(wm.config, 16 * ci + b), xp=torch, device=dev)
            psi_true[b] = torch.complex(-0.05 * phi, phi).to(torch.complex64)
        t = torch.from_numpy(S.diffuser(n, n, S.rng_for(wm.config, 99)).astype(np.complex64)).to(dev)
        f = plan.forward(psi_true, t)
        ph = torch.tensor([S.mixed_photons(wm.config, 16 * ci + b) for b in range(S.MIXED_PER_SIZE)],
                          dtype=torch.float32, device=dev)[:, None, None]
        g = torch.Generator(device=dev).manual_seed(20146500 + ci)
        y = (torch.poisson(f.clamp_min(0) * ph, generator=g) / ph).contiguous()
        plans.append(plan)
        ys.append(y)
        ts.append(t)
        psis.append(torch.zeros_like(psi_true))
        mpx += S.MIXED_PER_SIZE * n * n / 1e6
        del f, psi_true
    group = P.pwf_group_create(plans)
    P.pwf_group_solve(group, ys, ts, psis, 2)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for p in psis:
        p.zero_()
    P.pwf_group_solve(group, ys, ts, psis, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    shapes = [P.pwf_plan_describe(p.handle).split(" col_q")[0] for p in plans]
    # each size class alone (its own graph, whole GPU): where the group's time goes
    hbm, _ = peaks()
    per_class = []
    for ci, n in enumerate(S.MIXED_SIZES):
        plans[ci].solve(ys[ci], ts[ci], psis[ci], 1, read_back=False)
        torch.cuda.synchronize()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        plans[ci].solve(ys[ci], ts[ci], psis[ci], 2, read_back=False)
        c1.record(stream)
        torch.cuda.synchronize()
        cms = c0.elapsed_time(c1) / 2
        px = S.MIXED_PER_SIZE * n * n
        # per pass (event pairs around every kernel of one eager iteration):
        # total ms per pass name and each pass's algorithmic rate against the copy rate
        tot, cnt = {}, {}
        for name, pms in P.pwf_profile_iteration(plans[ci].handle, ys[ci], ts[ci], psis[ci], 1):
            tot[name] = tot.get(name, 0.0) + pms
            cnt[name] = cnt.get(name, 0) + 1
        frac = {name: round(PASS_BYTES_PER_PX[name] * px * cnt[name] / (tot[name] / 1e3) / 1e9 / hbm, 3)
                for name in tot if PASS_BYTES_PER_PX.get(name)}
        per_class.append({"n": n, "ms_per_iter_alone": cms,
                          "model_frac_of_measured_hbm": px * modal_bytes_per_px(wm.n_modes) / (cms / 1e3) / 1e9 / hbm,
                          "pass_ms": {k: round(v, 3) for k, v in sorted(tot.items(), key=lambda kv: -kv[1])},
                          "pass_frac_of_measured_hbm": frac})
    P.pwf_group_destroy(group)
    for p in plans:
        p.close()
    bpp = modal_bytes_per_px(wm.n_modes)
    gbs = mpx * 1e6 * bpp / (ms / steps / 1e3) / 1e9
    return {"value": mpx * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
            "workload": wm.name, "mpx_per_iter": mpx, "classes": shapes,
            "launch": "one CUDA graph launch per iteration over all four size classes",
            "model_bytes_per_px": bpp, "model_gbs": gbs, "model_frac_of_measured_hbm": gbs / hbm,
            "per_class_alone": per_class}


def run_small(P, S, torch, dev, stream, reps=5):
    """The single-projection workloads: 128^2 coherent (50 iterations) and
    512^2 with partial coherence (100 iterations; IOTF form and K = 9 source
    modes). One solve call of the workload's iterations is timed: the graph
    holding the loop (the default), the persistent cooperative launch and the
    cluster-resident launch (one thread-block cluster per projection; every
    cluster size that fits is timed, the default size gives the line). At these
    sizes an iteration is a chain of ~13 passes over a field that sits in L2:
    latency, not HBM, sets the time, so no HBM fraction is reported."""
    import numpy as np
    out = {}
    cases = (("blob128_coherent", 0), ("blob512_iotf", 0), ("blob512_iotf", 9))
    for name, K in cases:
        w = S.WORKLOADS[name]
        psi_true = torch.from_numpy(S.complex_phase_from(S.blob_phase(w.ny, w.nx, S.rng_for(w.config, 0)))
                                    .astype(np.complex64))[None].to(dev)
        t = torch.from_numpy(S.diffuser(w.ny, w.nx, S.rng_for(w.config, 99)).astype(np.complex64)).to(dev)
        paths = ((("graph", P.FLAG_GRAPH), ("graph_no_pdl", P.FLAG_GRAPH | P.FLAG_NO_PDL),
                  ("persistent", P.FLAG_PERSISTENT), ("cluster", P.FLAG_CLUSTER))
                 if K == 0 else (("graph", 0), ("graph_no_pdl", P.FLAG_NO_PDL)))

        def timed_solve(plan, y, psi):
            for _ in range(3):
                psi.zero_()
                plan.solve(y, t, psi, w.n_iter, read_back=False)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                psi.zero_()
                plan.solve(y, t, psi, w.n_iter, read_back=False)
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps

        for path, flags in paths:
            plan = P.Plan(P.PlanDesc(1, w.ny, w.nx, w.pixel_m, w.wavelength_m, w.L1_m, w.L2_m, w.xcoh_m, w.ycoh_m,
                                     w.gamma, w.alpha.real, w.alpha.imag, w.eta, flags, K, 2.0 if K else 0.0))
            f = plan.forward(psi_true, t)
            g = torch.Generator(device=dev).manual_seed(20146000 + 100 * w.config)
            y = (torch.poisson(f.clamp_min(0) * w.photons, generator=g) / w.photons).contiguous()
            psi = torch.zeros_like(psi_true)
            ms = timed_solve(plan, y, psi)
            key = f"{name}{'_k%d' % K if K else ''}_{path}"
            out[key] = {"value": w.ny * w.nx * w.n_iter / 1e6 / (ms / 1e3), "unit": UNIT,
                        "iterations_per_s": w.n_iter / (ms / 1e3), "us_per_iteration": 1e3 * ms / w.n_iter,
                        "ms_per_solve": ms, "iterations": w.n_iter, "ny": w.ny, "nx": w.nx, "n_modes": K,
                        "hbm_fraction": "not applicable (latency bound, field resident in L2)"}
            if path == "cluster":
                default, dsched = P.pwf_plan_cluster_size(plan.handle), P.pwf_plan_cluster_schedule(plan.handle)
                sweep = {}
                for sched in (0, 1):
                    try:
                        P.pwf_plan_set_cluster_schedule(plan.handle, sched)
                    except P.PWFError:
                        continue
                    for cs in (1, 2, 4, 8, 16):
                        try:
                            P.pwf_plan_set_cluster_size(plan.handle, cs)
                        except P.PWFError:
                            continue
                        sweep[f"set{sched}_{cs}"] = round(1e3 * timed_solve(plan, y, psi) / w.n_iter, 2)
                P.pwf_plan_set_cluster_schedule(plan.handle, dsched)
                P.pwf_plan_set_cluster_size(plan.handle, default)
                out[key].update({"cluster_ctas": default, "cluster_schedule_set": dsched,
                                 "schedule": P.pwf_plan_describe(plan.handle).split("cluster_schedule=")[1].split()[0],
                                 "us_per_iteration_by_schedule_set_and_ctas": sweep})
            plan.close()
    return out


def run_autograd(P, S, torch, dev, stream, reps=3):
    """Forward model + hand-written backward (w.r.t. psi and the diffuser) via
    the autograd Function, 16 projections of 2048^2, in the IOTF form and with
    25 source modes (mode fields recomputed in the backward, never stored)."""
    import numpy as np
    from paper_2503_20146_gb300.autograd import physical_model
    out = {}
    for name in ("grad16x2048_iotf", "grad16x2048_k25"):
        wg = S.WORKLOADS[name]
        plan = P.Plan(plan_desc(P, wg, wg.batch))
        psi = torch.empty((wg.batch, wg.ny, wg.nx), dtype=torch.complex64, device=dev)
        for b in range(wg.batch):
            phi = S.blob_phase(wg.ny, wg.nx, S.rng_for(wg.config, b), xp=torch, device=dev)
            psi[b] = torch.complex(-0.05 * phi, phi).to(torch.complex64)
        t = torch.from_numpy(S.diffuser(wg.ny, wg.nx, S.rng_for(wg.config, 99)).astype(np.complex64)).to(dev)
        wts = torch.randn(psi.shape, generator=torch.Generator(device=dev).manual_seed(4), device=dev)
        psi.requires_grad_(True)
        t.requires_grad_(True)

        def step():
            psi.grad = None
            t.grad = None
            (physical_model(psi, t, plan) * wts).sum().backward()

        step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        mpx = wg.batch * wg.ny * wg.nx / 1e6
        out[name] = {"ms_per_forward_backward": ms, "Mpx_per_s": mpx / (ms / 1e3), "n_modes": wg.n_modes}
        plan.close()
        del psi, t, wts
    return out


def run_fbp(P, S, torch, dev, stream, psi, w, reps=3):
    """Tomography after the path: filtered back projection (Ram-Lak, one slice
    per detector row) of the retrieved series into a ny x nx x nx volume."""
    n_ang, ny, nx = psi.shape
    angles = S.tomo_angles(n_ang)
    vol = torch.empty((ny, nx, nx), dtype=torch.complex64, device=dev)
    ws = torch.empty(P.pwf_fbp_workspace_bytes(n_ang, ny, nx), dtype=torch.uint8, device=dev)
    P.pwf_fbp(psi, angles, w.wavelength_m, w.pixel_m, vol, ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        P.pwf_fbp(psi, angles, w.wavelength_m, w.pixel_m, vol, ws)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    updates = float(n_ang) * ny * nx * nx
    out = {"ms": ms, "voxel_angle_updates_per_s": updates / (ms / 1e3), "volume": [ny, nx, nx],
           "angles": n_ang, "note": "includes the host-side ramp and angle tables (synchronous copies)"}
    del vol, ws
    return out


# ----------------------------------------------------------------------------
# main arm
# ----------------------------------------------------------------------------
def main():
    args = parse_args()
    from paper_2503_20146_gb300 import synth as S
    w = S.WORKLOADS[args.workload]
    rank, world, local = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, w, rank, world)
        return
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")

    import numpy as np
    import torch

    from paper_2503_20146_gb300 import _build
    if rank == 0:
        _build.build()
    barrier(world)
    from paper_2503_20146_gb300 import pwf as P
    P.load()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    batch = args.batch or w.batch
    mpx_iter = batch * w.ny * w.nx / 1e6

    psi_true, t = make_workload(P, S, w, batch, dev, rank, world)
    plan = P.Plan(plan_desc(P, w, batch))
    f = plan.forward(psi_true, t)
    gen = torch.Generator(device=dev).manual_seed(20146000 + 100 * w.config + rank)
    y = (torch.poisson(f.clamp_min(0) * w.photons, generator=gen) / w.photons).contiguous()
    del f, psi_true
    psi = torch.zeros((batch, w.ny, w.nx), dtype=torch.complex64, device=dev)

    if args.column_shapes:
        for op, k in enumerate(int(v) for v in args.column_shapes.split(",")):
            P.pwf_plan_set_column_shape(plan.handle, op, k)
    tuned = P.pwf_plan_describe(plan.handle)
    shape_ids = selected_shape_ids(tuned)

    # warm-up (captures the iteration graph)
    plan.solve(y, t, psi, args.warmup, read_back=False)
    torch.cuda.synchronize()

    # timed region: K iterations of Algorithm S1 (one pwf_solve call)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = P.pwf_plan_launch_count(plan.handle)
    with ClockSampler(local) as clk:
        barrier(world)
        torch.cuda.synchronize()
        e0.record(stream)
        psi.zero_()
        plan.solve(y, t, psi, args.steps, read_back=False)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        launches = P.pwf_plan_launch_count(plan.handle) - launches0
        # per-pass timing (eager, CUDA events around each kernel) -> roofline;
        # inside the sampled window too, since the roofline comes from it
        psi.zero_()
        passes = P.pwf_profile_iteration(plan.handle, y, t, psi, 3)
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    value = world * mpx_iter * args.steps / (ms / 1e3)

    hbm, peak_kind = peaks()
    tot = {}
    for name, pms in passes:
        tot[name] = tot.get(name, 0.0) + pms
    dom = max(tot, key=tot.get)
    dom_ms = [pms for name, pms in passes if name == dom]
    dom_avg = sum(dom_ms) / len(dom_ms)
    dom_bytes = PASS_BYTES_PER_PX.get(dom, 0) * batch * w.ny * w.nx
    achieved = dom_bytes / (dom_avg / 1e3) / 1e9
    iter_ms = sum(p for _, p in passes)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": measured_traffic(dom), "peak_kind": peak_kind,
                "bytes_per_px": PASS_BYTES_PER_PX.get(dom, 0), "launch_ms": dom_avg,
                "share_of_iteration": sum(dom_ms) / iter_ms}
    # the same launch against the instruction issue rate (the column passes are
    # issue-bound): instruction count from the ncu capture, clock sampled above
    try:
        ipx = measured_instructions_per_px(dom)
        clk_mhz = clk.summary().get("sm_mhz") or max_sm_mhz()
        if ipx is not None and clk_mhz:
            sms = torch.cuda.get_device_properties(dev).multi_processor_count
            roofline["issue"] = issue_roofline(ipx, batch * w.ny * w.nx, dom_avg, sms, clk_mhz)
    except Exception as exc:  # an auxiliary figure never costs the bench line
        roofline["issue"] = {"unavailable": repr(exc)}
    model_bytes = sum(PASS_BYTES_PER_PX.get(n, 0) for n, _ in passes) * batch * w.ny * w.nx
    iteration = {"passes": [[n, round(p, 4)] for n, p in passes],
                 "eager_iteration_ms": iter_ms,
                 "model_bytes_per_px": sum(PASS_BYTES_PER_PX.get(n, 0) for n, _ in passes),
                 "model_gbs_timed": model_bytes / (ms / args.steps / 1e3) / 1e9,
                 "model_frac_timed": model_bytes / (ms / args.steps / 1e3) / 1e9 / hbm,
                 # what the method must touch once per iteration (psi r/w, phi r/w, t, y):
                 # the bound if a whole field stayed on chip
                 "state_floor_bytes_per_px": STATE_FLOOR_BYTES_PER_PX,
                 "state_floor_frac_timed": STATE_FLOOR_BYTES_PER_PX * batch * w.ny * w.nx
                 / (ms / args.steps / 1e3) / 1e9 / hbm}

    extras = {}
    legs = set(args.legs.split(",")) if args.legs != "all" else None

    def leg(name):
        return legs is None or name in legs

    if not args.no_extras and leg("e2e"):
        # end to end through the host-buffer entry point, every rank on its own
        # series: y and t from pinned host memory, psi (from 0) back to it;
        # chunks of the series stream through the device with the copies
        # overlapping the solve. Barrier before each call, max over ranks.
        e2e_iters = 10
        y_h = y.cpu().pin_memory()
        t_h = t.cpu().pin_memory()
        psi_h = torch.empty(psi.shape, dtype=psi.dtype).pin_memory()
        times = []
        for rep in range(3):  # the first call builds the chunk plans
            torch.cuda.synchronize()
            barrier(world)
            t0 = time.perf_counter()
            plan.solve_host(y_h, t_h, psi_h, e2e_iters, psi_is_input=False)
            dt = max_over_ranks(time.perf_counter() - t0, world)
            if rep > 0:
                times.append(dt * 1e3)
        ems = sum(times) / len(times)
        chunk = [c for c in range(-(-batch // 4), 0, -1) if batch % c == 0][0]
        extras["e2e"] = {"value": world * mpx_iter * e2e_iters / (ems / 1e3), "unit": UNIT,
                         "h2d_bytes_per_step": int(world * (y.numel() * 4 + t.numel() * 8)),
                         "d2h_bytes_per_step": int(world * psi.numel() * 8),
                         "step": f"one pwf_solve_host call of {e2e_iters} iterations per rank (pinned host "
                                 f"buffers, chunks of {chunk} projections, copies overlapping the solve)",
                         "ms_per_call": ems}
        del y_h, t_h, psi_h

    if not args.no_extras and rank == 0:
        if leg("plain"):
            # plain per-projection baseline (unfused, Algorithm S2 step by step) on a sample
            nplain, iplain = 16, 5
            plain = P.Plan(plan_desc(P, w, nplain, P.FLAG_PLAIN))
            yp = y[:nplain].contiguous()
            pp = torch.zeros((nplain, w.ny, w.nx), dtype=torch.complex64, device=dev)
            plain.solve(yp, t, pp, 1, read_back=False)
            torch.cuda.synchronize()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            pp.zero_()
            plain.solve(yp, t, pp, iplain, read_back=False)
            a1.record(stream)
            torch.cuda.synchronize()
            pv = nplain * w.ny * w.nx * iplain / 1e6 / (a0.elapsed_time(a1) / 1e3)
            extras["plain_gpu"] = {"value": pv, "unit": UNIT, "sample": f"{nplain} projections x {iplain} iterations",
                                   "fused_over_plain": value / world / pv}
            plain.close()
            del yp, pp

        # the same series with partial coherence as 9 tilted source modes
        if leg("modal") and w.name == "tomo180x1024_iotf":
            wk = S.WORKLOADS["tomo180x1024_k9"]
            mplan = P.Plan(plan_desc(P, wk, batch))
            pm = torch.zeros_like(psi)
            mplan.solve(y, t, pm, 3, read_back=False)
            torch.cuda.synchronize()
            m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            msteps = 5
            m0.record(stream)
            pm.zero_()
            mplan.solve(y, t, pm, msteps, read_back=False)
            m1.record(stream)
            torch.cuda.synchronize()
            mms = m0.elapsed_time(m1)
            mbpp = modal_bytes_per_px(wk.n_modes)
            mgbs = batch * w.ny * w.nx * mbpp / (mms / msteps / 1e3) / 1e9
            pm.zero_()
            mpasses = P.pwf_profile_iteration(mplan.handle, y, t, pm, 1)
            mtot = {}
            for name, pms in mpasses:
                mtot[name] = mtot.get(name, 0.0) + pms
            mdom = max(mtot, key=mtot.get)
            mdom_ms = [pms for name, pms in mpasses if name == mdom]
            mdom_avg = sum(mdom_ms) / len(mdom_ms)
            mach = PASS_BYTES_PER_PX.get(mdom, 0) * batch * w.ny * w.nx / (mdom_avg / 1e3) / 1e9
            extras["modal_k9"] = {"metric": METRIC, "value": mpx_iter * msteps / (mms / 1e3), "unit": UNIT,
                                  "ms_per_step": mms / msteps, "workload": wk.name, "steps": msteps,
                                  "config": {"workload": wk.name, "projections_per_gpu": batch, "ny": w.ny,
                                             "nx": w.nx, "coherence": "9 source modes, sigma = 2 px"},
                                  "model_bytes_per_px": mbpp, "model_gbs": mgbs, "model_frac_of_measured_hbm": mgbs / hbm,
                                  "roofline": {"bound": "hbm", "kernel": mdom, "achieved": mach, "peak": hbm,
                                               "unit": "GB/s", "frac": mach / hbm, "traffic": None,
                                               "peak_kind": peak_kind, "launch_ms": mdom_avg,
                                               "share_of_iteration": sum(mdom_ms) / sum(p for _, p in mpasses)},
                                  "passes": [[n, round(x, 4)] for n, x in mpasses]}
            mplan.close()
            del pm

        # the single-projection workloads (128^2 coherent, 512^2 partially coherent)
        if leg("small") and w.name == "tomo180x1024_iotf":
            extras["small"] = run_small(P, S, torch, dev, stream)

        # uneven batch: 16 each of 256^2, 768^2, 1536^2, 2048^2, 25 modes, one group
        if leg("mixed") and w.name == "tomo180x1024_iotf":
            extras["mixed_k25"] = run_mixed(P, S, torch, dev, stream)

        # differentiation: 16 x 2048^2 forward + backward through torch.autograd
        if leg("autograd") and w.name == "tomo180x1024_iotf":
            extras["autograd_16x2048"] = run_autograd(P, S, torch, dev, stream)

        # tomography after the path: FBP of the retrieved series
        if leg("fbp") and w.name == "tomo180x1024_iotf":
            extras["fbp_180x1024"] = run_fbp(P, S, torch, dev, stream, psi, w)

        # ablations on a small synthetic series (preconditioner, gamma, alpha): PWF + FBP + scores
        if leg("ablation") and w.name == "tomo180x1024_iotf":
            from paper_2503_20146_gb300 import ablation as A
            series = A.make_series(n_angles=32, n=128)
            extras["ablation_32x128"] = {"iterations": 150, "rows": A.run_ablation(series, iters=150)}
            del series

        if leg("cpu"):
            # FP64 oracle on every host core (one worker process per core, each
            # on its own projection), bounded sample (~10 s of CPU work per core)
            pool = OraclePool()
            pool.sample(w, 1)  # workers start and import numpy
            dt, work = pool.sample(w, CPU_SAMPLE_ITERS)
            extras["cpu_baseline"] = {"value": work / dt, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
                                      "sample": f"{pool.cores} projections of {w.ny}x{w.nx} (one per core), "
                                                f"{CPU_SAMPLE_ITERS} iterations, numpy FP64",
                                      "seconds": dt}
            pool.close()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "projections_per_gpu": batch, "ny": w.ny, "nx": w.nx,
                       "coherence": "IOTF, Gaussian sigma = 2 px" if w.xcoh_m > 0 else "coherent",
                       "eta": w.eta, "l2_flush": "inputs larger than L2 (state ~1.5 GB per field)",
                       "step": "one PWF iteration over all projections",
                       "column_shapes": tuned, "column_shape_ids": shape_ids},
            "gpu_launches": int(launches),
            "roofline": roofline,
            "iteration": iteration,
            "clocks": clk.summary(),
        }
        line.update(extras)
        if "e2e" not in line:
            line["e2e"] = None
        print(json.dumps(line))
    plan.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
