#!/usr/bin/env python3
"""Throughput of the PCEXP Krylov step on GB300: DOF * steps / s.

Workload (headline): the 3D isentropic vortex (axis along z) on the periodic cube
[0,10]^3, 48^3 cubes split into 663,552 Kuhn tetrahedra with +-10% node jitter
(seed 5), DG P2 (K = 33,177,600 unknowns), Ma 0.5 at 45 degrees, PCEXP with the
global time step at CFL 10 and Krylov dimension m = 30, started from the projected
vortex.  One step = one PCEXP step (residual, point Jacobians, two CGS2 Arnoldi
processes of 30 columns with their J v products, two phi evaluations, the corrector
residual and J v, both updates).  The headline value is the FP32-mixed form; the
FP64 form runs the same steps beside it and the FP32-mixed state error against it
is stated.  The 2D bump channel (192 x 64, P2, local CFL 100) is a side block.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
For N > 1 run under torchrun; every rank runs an independent replica (the path is
not sharded across GPUs here), so the scaling is weak.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "PCEXP DOF·steps/s on DG Euler, FP32-mixed vs FP64 at stated error, % HBM peak"
UNIT = "DOF*steps/s"
N3D, P3D, M3D, CFL3D = 48, 2, 30, 10.0
WORKLOAD = f"vortex3d_{N3D}cubed_kuhn_p{P3D}_m{M3D}_pcexp_globalcfl10"
# bounded CPU samples of the same configuration (smaller cubes of the same vortex)
CPU_SAMPLE_N, CPU_SAMPLE_STEPS = 6, 3
REF_SAMPLE_N = 4
# 2D side block (the steady bump channel with local time steps)
NX, NY, P2D, M2D, CFL2D, SEED2D = 192, 64, 2, 30, 100.0, 1


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------------- CPU oracle
ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import workloads as W
from oracle.dg import DGOracle
from oracle import pcexp
from oracle.cases import vortex_state
case = W.case_vortex3d(n={n})
dg = DGOracle(case.mesh, case.p, case.free)
u = dg.project(lambda x: vortex_state(x, case.free, case.vortex, period=10.0)).reshape(-1)
times = []
for s in range({warm} + {steps}):
    t0 = time.perf_counter()
    dt = float(np.min(dg.local_dt(u, case.cfl)))
    u, _ = pcexp.pcexp_step(u, dg.residual, dg.jvp, dt, case.m)
    times.append(time.perf_counter() - t0)
print(json.dumps(dict(K=dg.K, E=dg.E, times=times[{warm}:])))
"""


def run_oracle(n, steps, warm):
    """The FP64 oracle, single-threaded, on the n^3 sample of the 3D vortex: per-step times."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ORACLE_SNIPPET.format(root=ROOT, n=n, warm=warm, steps=steps)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed:\n" + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


# ------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.dev = device_index

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------ algorithmic bytes
def shape(dim, p):
    """(nb, nq, nfq, nv, nf): basis size, volume and face points, variables, faces per element."""
    if dim == 2:
        return (p + 1) * (p + 2) // 2, (p + 1) ** 2, p + 1, 4, 3
    if p == 2:  # the symmetric rules of tetrahedra at p = 2
        return 10, 14, 7, 5, 4
    return (p + 1) * (p + 2) * (p + 3) // 6, (p + 1) ** 3, (p + 1) ** 2, 5, 4


def second_pass_columns(masks, m):
    """(fraction of the Gram-Schmidt update-and-norm launches that ran, mean column index of
    those that ran) from the step infos' reorth_cols bit masks (bit j: column j of a stage ran
    the second pass; the other launches of the class leave at once)."""
    ran = [j for mk in masks for j in range(m) if (mk >> j) & 1]
    if not masks:
        return 1.0, (m - 1) / 2.0
    return len(ran) / (m * len(masks)), (sum(ran) / len(ran) if ran else 0.0)


def algorithmic_bytes(kind, T, K, E, F, dim, p, m, face_jacobians=True, gs=None):
    """DRAM bytes per launch of a kernel class: every input it needs read once and every
    output written once (T = 4 or 8 bytes per value).  G is the face-flux buffer
    [F][nfq][nv] between the face and element kernels of one operator application.

    jvp: one whole J v application (face + element kernels) at its minimum of three
    K-vector passes (read v, read the linearisation state, write J v) plus the element
    geometry, the figure a fused J v would move.  gs = second_pass_columns(...): the
    update-and-norm class counts the columns that ran the second pass only (averaged over
    the class's launches)."""
    nb, nq, nfq, nv, nf = shape(dim, p)
    geo = dim * dim + 3
    g_face = F * ((dim + 1) * T + 12)  # normal, measure, element and local-face ids
    g_elem = E * (geo * T + 4 * nf)    # inverse map, sqrt(det), h, 1/sqrt(det); face slots
    G = F * nfq * nv * T
    avg_j = (m - 1) / 2.0              # mean column index over one Arnoldi process
    if T == 8:   # FP64: the volume part applies the stored point Jacobians
        jvp_elem = 2 * K * T + dim * nv * nv * E * nq * T + E * (T + 4 * nf) + G
    else:        # FP32-mixed: flux tangents recomputed from the linearisation state
        jvp_elem = 3 * K * T + g_elem + G
    if face_jacobians:  # face point Jacobians at u_n (both sides) applied to the traces of v
        jvp_face = K * T + 2 * nv * nv * F * nfq * T + F * 12 + G
    else:               # Riemann-flux tangents recomputed from the traces of u_n and v
        jvp_face = 2 * K * T + g_face + G
    return {
        "jvp_face": jvp_face,
        "jvp_elem": jvp_elem,
        "jvp": 3 * K * T + g_elem,
        "residual_face": K * T + g_face + G,
        "residual_elem": 2 * K * T + g_elem + G,
        "cgs_proj": (avg_j + 2) * K * T,
        "cgs_upd_proj": (avg_j + 3) * K * T,
        "cgs_upd_norm": (gs[0] * (gs[1] + 3) if gs else avg_j + 3) * K * T,
        "cgs_upd1": (avg_j + 3) * K * T,
        "cgs_proj2": (gs[0] * (gs[1] + 2) if gs else avg_j + 2) * K * T,
    }.get(kind)


def algorithmic_flops(kind, K, E, F, dim, p, m, T=8, gs=None):
    """Floating-point operations per launch of a kernel class (an FMA counts 2).

    jvp_elem, FP64 (stored point Jacobians): per element, nq points x (trace nv nb + Jacobian
    d nv^2) FMA and nv nb outputs x (volume d nq + lift nf nfq) FMA.  FP32-mixed (flux
    tangents): nq points x (traces of u_n and v, 2 nv nb; mapping of the flux tangent to
    reference directions, d^2 nv) FMA and the same test and lift; the Euler-flux tangent itself
    (a few hundred operations per point) is not counted, so the fraction is a lower bound.
    jvp_face: per face point 2 nv nb trace + 2 nv^2 FMA; CGS kernels: per unknown and column,
    1 (projection) or 2 (update + projection) FMA, averaged over the columns of one Arnoldi
    process."""
    nb, nq, nfq, nv, nf = shape(dim, p)
    nc = (m + 1) / 2.0
    vol = nq * (nv * nb + dim * nv * nv) if T == 8 else nq * (2 * nv * nb + dim * dim * nv)
    fma = {
        "jvp_elem": E * (vol + nv * nb * (dim * nq + nf * nfq)),
        "jvp_face": F * nfq * (2 * nv * nb + 2 * nv * nv),
        "cgs_proj": K * (nc + 1),
        "cgs_upd_proj": K * 2 * nc,
        "cgs_upd_norm": K * (gs[0] * (gs[1] + 2) if gs else nc + 1),
        "cgs_upd1": K * (nc + 1),
        "cgs_proj2": K * (gs[0] * (gs[1] + 2) if gs else nc + 1),
    }.get(kind)
    return None if fma is None else 2.0 * fma


# DRAM bytes (read + write) per launch from one ncu capture of the same kernel on the same
# workload, keyed (workload, element bytes, kernel class); an entry is dropped when its
# kernel changes.  The summaries under profiles/ give the commands.
NCU_TRAFFIC = {
    ("vortex3d", 4, "jvp_elem"): (608250112, "profiles/traffic_vortex3d_48_p2_m30_fp32.md"),
}


def fp64_peak(capi):
    """Measured FP64 FMA rate (TFLOP/s) of this GPU from the library's DFMA-chain kernel."""
    try:
        return capi.fp64_fma_rate(), "measured: DFMA chains on every SM, CUDA events"
    except Exception:
        return 152 * 2 * 2 * 2.070e9 / 1e12, "derived: 152 SMs x 2 DFMA/clk x 2 x 2.07 GHz"


def fp32_peak(capi):
    """Measured FP32 FMA rate (TFLOP/s) of this GPU from the library's FFMA-chain kernel."""
    try:
        return capi.fp32_fma_rate(), "measured: FFMA chains on every SM, CUDA events"
    except Exception:
        return 152 * 128 * 2 * 2.070e9 / 1e12, "derived: 152 SMs x 128 FFMA/clk x 2 x 2.07 GHz"


def roofline_entry(prof, T, K, E, F, hbm, peak_kind, dim, p, m, workload, fp64=None, face_jacobians=True,
                   fp32=None, gs=None):
    """Roofline of the dominant kernel class by device time, against the roof that bounds it:
    the one with the longer minimum time, algorithmic bytes at the measured HBM copy rate or
    algorithmic flops at the measured FMA rate of its precision (FP64 pipe for FP64 kernels,
    FP32 FMA for FP32 ones).  Both fractions are given.  Adds the whole J v application
    (face + element time) against the three-K-pass minimum."""
    dom = max(prof, key=lambda k: prof[k][1])
    n_dom, ms_dom = prof[dom]
    if not n_dom:
        return None
    sec = ms_dom / n_dom / 1e3
    tr = NCU_TRAFFIC.get((workload, T, dom))
    entry = {"kernel": dom, "avg_launch_us": round(sec * 1e6, 2),
             "time_share": round(ms_dom / sum(v[1] for v in prof.values()), 4),
             "traffic": tr[0] if tr else None}
    if tr:
        entry["traffic_source"] = tr[1]
    ab = algorithmic_bytes(dom, T, K, E, F, dim, p, m, face_jacobians, gs)
    if ab is not None:
        entry["algorithmic_bytes_per_launch"] = ab
    fl = algorithmic_flops(dom, K, E, F, dim, p, m, T, gs)
    alu = fp64 if T == 8 else fp32
    t_alu = fl / (alu[0] * 1e12) if fl is not None and alu is not None else 0.0
    t_hbm = ab / (hbm * 1e9) if ab is not None else 0.0
    if t_alu > t_hbm:
        ach = fl / sec / 1e12
        entry.update({"bound": "alu", "achieved": round(ach, 3), "peak": round(alu[0], 3),
                      "unit": "TFLOP/s", "frac": round(ach / alu[0], 4),
                      "peak_source": ("FP64 FMA " if T == 8 else "FP32 FMA ") + alu[1],
                      "algorithmic_flops_per_launch": fl,
                      "hbm_frac": round(ab / sec / 1e9 / hbm, 4) if ab else None})
    elif ab is not None:
        ach = ab / sec / 1e9
        entry.update({"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                      "frac": round(ach / hbm, 4), "peak_source": peak_kind})
        if t_alu:
            entry["alu_frac"] = round(fl / sec / 1e12 / alu[0], 4)
    nf_, tf_ = prof.get("jvp_face", (0, 0.0))
    ne_, te_ = prof.get("jvp_elem", (0, 0.0))
    if ne_:
        sec_j = (tf_ + te_) / ne_ / 1e3
        bj = algorithmic_bytes("jvp", T, K, E, F, dim, p, m)
        entry["jvp_application"] = {"avg_us": round(sec_j * 1e6, 2), "bytes": bj,
                                    "gbs": round(bj / sec_j / 1e9, 1), "frac": round(bj / sec_j / 1e9 / hbm, 4)}
    return entry


def kernel_table(prof, T, K, E, F, hbm, dim, p, m, fp64=None, face_jacobians=True, fp32=None, gs=None):
    """Every kernel class with a byte model: launches, mean launch time (CUDA events per
    class over the profiled steps), algorithmic GB/s and its fraction of measured HBM;
    classes with a flop model also give TFLOP/s and the fraction of the measured FMA rate of
    their precision."""
    out = {}
    for kind, (n, ms) in prof.items():
        ab = algorithmic_bytes(kind, T, K, E, F, dim, p, m, face_jacobians, gs)
        if not n or ab is None:
            continue
        sec = ms / n / 1e3
        row = {"launches": n, "avg_launch_us": round(sec * 1e6, 2), "gbs": round(ab / sec / 1e9, 1),
               "hbm_frac": round(ab / sec / 1e9 / hbm, 4)}
        if kind in ("cgs_upd_norm", "cgs_proj2") and gs:
            row["ran"] = round(gs[0], 4)  # share of the launches that ran the second pass
        fl = algorithmic_flops(kind, K, E, F, dim, p, m, T, gs)
        if T == 8 and fl is not None and fp64 is not None:
            row["fp64_tflops"] = round(fl / sec / 1e12, 3)
            row["fp64_frac"] = round(fl / sec / 1e12 / fp64[0], 4)
        elif T == 4 and fl is not None and fp32 is not None:
            row["fp32_tflops"] = round(fl / sec / 1e12, 3)
            row["fp32_frac"] = round(fl / sec / 1e12 / fp32[0], 4)
        out[kind] = row
    return out


def step_hbm(prof, T, K, E, F, hbm, dim, p, m, ms_per_step, face_jacobians=True, gs=None):
    """The whole step against the HBM copy rate: the algorithmic bytes of every kernel class
    with a byte model, times its launches per step, over the device-timed step.  Classes bound
    by arithmetic (the element J v in FP32-mixed, the FP64 form) keep the step below 1."""
    total = 0.0
    for kind, (n, _ms) in prof.items():
        ab = algorithmic_bytes(kind, T, K, E, F, dim, p, m, face_jacobians, gs)
        if n and ab is not None:
            total += n * ab
    gbs = total / (ms_per_step / 1e3) / 1e9
    return {"algorithmic_bytes_per_step": total, "gbs": round(gbs, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(gbs / hbm, 4)}


def max_over_ranks(x, dist, device="cuda"):
    """The largest of the ranks' values of x (the slowest rank sets the job's time); x itself
    without a process group.  The tensor lives on `device` (cuda for NCCL, cpu for gloo)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank_step, steps, world, seconds):
    """Whole-job DOF * steps / s: every rank advances its own replica by `steps` steps of
    `units_per_rank_step` unknowns; `seconds` is the max over ranks."""
    return units_per_rank_step * steps * world / seconds


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 form of the headline workload")
    ap.add_argument("--no-2d", action="store_true", help="skip the 2D bump-channel side block")
    ap.add_argument("--no-two-pass", action="store_true",
                    help="skip the FP32-mixed run with both Gram-Schmidt passes on every column")
    ap.add_argument("--no-partitioned", action="store_true",
                    help="skip the side block of the headline workload split into element partitions")
    ap.add_argument("--n3d", type=int, default=N3D, help="cubes per side of the 3D vortex (profiling runs)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        return reference_arm(args, rank, world)

    import numpy as np
    import torch

    import workloads as W
    from paper_1801_06300_gb300 import build, capi

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        build()
    if dist:
        dist.barrier()
    capi.load()
    hbm, peak_kind = load_peaks()
    fp64 = fp64_peak(capi)
    fp32 = fp32_peak(capi)

    case = W.case_vortex3d(n=args.n3d)
    prm = [case.vortex.eps, *case.vortex.center, 10.0]
    E = case.mesh.n_elem
    F = 2 * E  # periodic: every face interior, shared by two elements

    def step(ctx):
        ctx.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GLOBAL_CFL, case.cfl, case.m, info=False)

    def timed(ctx, steps, clocks=False):
        """`steps` steps between a barrier + synchronize on both sides, one CUDA-event pair per
        step on torch's current stream (the context's stream).  Inputs are far larger than L2
        (a 133 MB FP32 state, a 4.1 GB Krylov basis), so no flush between steps."""
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(local) if clocks else None
        if sampler:
            sampler.start()
        for s in range(steps):
            evs[s][0].record()
            step(ctx)
            evs[s][1].record()
        torch.cuda.synchronize()
        ck = sampler.stop() if sampler else None
        if dist:
            dist.barrier()
        return sum(a.elapsed_time(b) for a, b in evs), ck

    def profiled(ctx, steps):
        """Per-class CUDA-event times of `steps` steps, and the steps' second-pass column masks."""
        ctx.profile_enable(True)
        masks = []
        for _ in range(steps):
            info = ctx.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GLOBAL_CFL, case.cfl, case.m)
            masks += list(info["reorth_cols"])
        torch.cuda.synchronize()
        prof = ctx.profile_read()
        ctx.profile_enable(False)
        return prof, masks

    forms = {}
    order = [("fp32_mixed", capi.PCEXP_FP32_MIXED)] + ([] if args.no_fp64 else [("fp64", capi.PCEXP_FP64)])
    ctx32 = None
    for name, prec in order:
        ctx = capi.Context(case.mesh, case.p, case.free, prec, m_max=case.m)
        ctx.project_state(capi.PCEXP_PROJ_VORTEX, prm)
        for _ in range(args.warmup):
            step(ctx)
        torch.cuda.synchronize()
        ms, clocks = timed(ctx, args.steps, clocks=True)
        ms = max_over_ranks(ms, dist)
        state = ctx.get_state()
        nprof = 1 if name == "fp64" else 2
        prof, masks = profiled(ctx, nprof)
        prof = {k: (v[0] / nprof, v[1] / nprof) for k, v in prof.items()}  # per step
        gs = second_pass_columns(masks, case.m)
        T = 4 if name == "fp32_mixed" else 8
        forms[name] = {
            "value": job_throughput(ctx.K, args.steps, world, ms / 1e3), "ms_per_step": ms / args.steps,
            "state": state, "clocks": clocks, "prof": prof,
            "kernel_ms_per_step": {k: round(v[1], 4) for k, v in prof.items() if v[0]},
            "roofline": roofline_entry(prof, T, ctx.K, E, F, hbm, peak_kind, 3, case.p, case.m, "vortex3d", fp64,
                                       fp32=fp32, gs=gs),
            "kernels": kernel_table(prof, T, ctx.K, E, F, hbm, 3, case.p, case.m, fp64, fp32=fp32, gs=gs),
            "step_hbm": step_hbm(prof, T, ctx.K, E, F, hbm, 3, case.p, case.m, ms / args.steps, gs=gs),
            "gram_schmidt": {"reorth": "selective" if T == 4 else "always",
                             "second_pass_columns": f"{sum(bin(x).count('1') for x in masks)} of "
                                                    f"{case.m * len(masks)} (profiled steps)"},
        }
        if name == "fp32_mixed":
            ctx32 = ctx
        else:
            ctx.close()
    K = ctx32.K
    head = forms["fp32_mixed"]
    launches_per_step = sum(v[0] for v in head["prof"].values())

    # the FP32-mixed form with both Gram-Schmidt passes on every column (CGS2), the same steps
    two_pass = None
    if not args.no_two_pass:
        ctx = capi.Context(case.mesh, case.p, case.free, capi.PCEXP_FP32_MIXED, m_max=case.m,
                           reorth=capi.PCEXP_REORTH_ALWAYS)
        ctx.project_state(capi.PCEXP_PROJ_VORTEX, prm)
        for _ in range(args.warmup):
            step(ctx)
        torch.cuda.synchronize()
        ms2, _ = timed(ctx, args.steps)
        ms2 = max_over_ranks(ms2, dist)
        u2 = ctx.get_state()
        ctx.close()
        two_pass = {"ms_per_step": ms2 / args.steps, "value": job_throughput(K, args.steps, world, ms2 / 1e3),
                    "selective_speedup": ms2 / args.steps / head["ms_per_step"],
                    "state_rel_diff_vs_selective": float(np.linalg.norm(u2 - head["state"]) /
                                                         np.linalg.norm(head["state"]))}
        if "fp64" in forms:
            a = forms["fp64"]["state"]
            two_pass["state_rel_l2_vs_fp64"] = float(np.linalg.norm(u2 - a) / np.linalg.norm(a))

    # end to end through the public API with host buffers: every step copies the state in from
    # pinned host memory, steps, and copies it back out (copies inside the timed region)
    hin = torch.empty(K, dtype=torch.float64, pin_memory=True).numpy()
    hout = torch.empty(K, dtype=torch.float64, pin_memory=True).numpy()
    ctx32.get_state(hin)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx32.set_state(hin)
        step(ctx32)
        ctx32.get_state(hout)
        hin, hout = hout, hin
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist)
    # the state transfer alone (copy in from pinned host memory with the basis conversion, and
    # out again), by the wall clock around the synchronising calls
    t0 = time.perf_counter()
    for _ in range(5):
        ctx32.set_state(hin)
    set_ms = (time.perf_counter() - t0) / 5 * 1e3
    t0 = time.perf_counter()
    for _ in range(5):
        ctx32.get_state(hout)
    get_ms = (time.perf_counter() - t0) / 5 * 1e3
    ctx32.close()

    err = None
    if "fp64" in forms:
        a, b = forms["fp64"]["state"], head["state"]
        err = float(np.linalg.norm(b - a) / np.linalg.norm(a))

    side = None if args.no_2d else bump2d_block(args, capi, W, torch, np, hbm, peak_kind, fp64, dist, fp32)
    parted = None if (args.no_partitioned or world > 1) else partitioned_block(args, capi, case, prm, np, torch)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = run_oracle(CPU_SAMPLE_N, steps=CPU_SAMPLE_STEPS, warm=0)
        cpu = {"value": r["K"] * len(r["times"]) / sum(r["times"]), "unit": UNIT, "cores": 1,
               "nproc": os.cpu_count(), "kind": "oracle",
               "sample": f"{CPU_SAMPLE_STEPS} PCEXP steps of the same configuration (vortex, P2, m = 30, "
                         f"CFL 10) on {CPU_SAMPLE_N}^3 cubes = {r['E']} tetrahedra (K = {r['K']}), FP64 numpy "
                         f"oracle, 1 thread of {os.cpu_count()}, {sum(r['times']):.1f} s"}

    def strip(f):
        return {k: v for k, v in f.items() if k not in ("state", "prof")}

    out = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD if args.n3d == N3D else f"vortex3d_{args.n3d}cubed_kuhn_p2_m30",
                   "mesh": f"{args.n3d}^3 cubes, {E:,} Kuhn tetrahedra, 10% jitter seed 5, periodic [0,10]^3",
                   "p": case.p, "m": case.m, "K": K, "scheme": "PCEXP", "time_step": "global, CFL 10",
                   "precision": "FP32-mixed (R, J v, Krylov basis FP32; reductions, H, phi, state FP64)",
                   "l2": "not flushed: inputs far larger than L2 (133 MB FP32 state, 4.1 GB Krylov basis)",
                   "parallelism": f"replicas x{world}"},
        "fp32_state_rel_l2_vs_fp64": err,
        "fp32_error_note": (f"relative L2 difference of the FP32-mixed and FP64 states after the same "
                            f"{args.warmup + args.steps} steps from the projected vortex"),
        "e2e": {"value": job_throughput(K, args.steps, world, e2e_s), "unit": UNIT,
                "h2d_bytes_per_step": K * 8, "d2h_bytes_per_step": K * 8,
                "ms_per_step": e2e_s / args.steps * 1e3, "set_state_ms": set_ms, "get_state_ms": get_ms},
        "gpu_launches": int(launches_per_step * args.steps),
        "roofline": head["roofline"],
        "fma_peaks": {"fp64_tflops": round(fp64[0], 3), "fp64_source": fp64[1],
                      "fp32_tflops": round(fp32[0], 2), "fp32_source": fp32[1]},
        "kernel_ms_per_step": head["kernel_ms_per_step"],
        "kernels": head["kernels"],
        "step_hbm": head["step_hbm"],
        "fp64": strip(forms["fp64"]) if "fp64" in forms else None,
        "speedup_fp32_mixed_vs_fp64": (forms["fp64"]["ms_per_step"] / head["ms_per_step"]) if "fp64" in forms else None,
        "gram_schmidt": head["gram_schmidt"],
        "fp32_mixed_two_pass": two_pass,
        "cpu_baseline": cpu,
        "bump2d": side,
        "partitioned": parted,
        "clocks": head["clocks"],
    }
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def partitioned_block(args, capi, case, prm, np, torch, n_parts=2, steps=5, warm=2):
    """Side block: the headline workload split into n_parts element partitions (recursive
    coordinate bisection, one-element halos), all on this GPU, FP32-mixed, against one context
    on the whole mesh, both driven through the public API with per-step host synchronisation
    (step info read back) and timed by the wall clock over the same steps.  Reports both times
    and the relative state difference after the same steps (the partitions' split
    Gram-Schmidt sums round differently)."""
    part = capi.partition(case.mesh, n_parts)

    def run(make):
        obj = make()
        obj.project_state(capi.PCEXP_PROJ_VORTEX, prm)
        for _ in range(warm):
            obj.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GLOBAL_CFL, case.cfl, case.m)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            obj.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GLOBAL_CFL, case.cfl, case.m)
        torch.cuda.synchronize()
        sec = (time.perf_counter() - t0) / steps
        u = obj.get_state()
        obj.close()
        return sec, u

    t_g, u_g = run(lambda: capi.Group(case.mesh, part, case.p, case.free, capi.PCEXP_FP32_MIXED, m_max=case.m))
    t_1, u_1 = run(lambda: capi.Context(case.mesh, case.p, case.free, capi.PCEXP_FP32_MIXED, m_max=case.m))
    K = u_1.size
    return {"parts": n_parts, "devices": [0] * n_parts, "steps": steps, "warmup": warm,
            "ms_per_step": t_g * 1e3, "value": K / t_g, "unit": UNIT,
            "single_context_ms_per_step": t_1 * 1e3, "time_vs_single_context": t_g / t_1,
            "state_rel_diff_vs_single_context": float(np.linalg.norm(u_g - u_1) / np.linalg.norm(u_1)),
            "timing": "wall clock, per-step host synchronisation, the same for both"}


def bump2d_block(args, capi, W, torch, np, hbm, peak_kind, fp64, dist=None, fp32=None):
    """Side block: the steady bump channel (192 x 64 split quads, 24,576 triangles, P2, local
    CFL 100, m = 30) in both forms, with a 256 MB L2 flush before each step (its vectors are
    L2-sized) outside the step's CUDA events."""
    case = W.case_bump2d(NX, NY, P2D, SEED2D)
    steps = max(3, min(args.steps, 10))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    E = case.mesh.n_elem
    F = (3 * E + len(case.mesh.btags)) // 2
    res = {}
    for name, prec in (("fp64", capi.PCEXP_FP64), ("fp32_mixed", capi.PCEXP_FP32_MIXED)):
        ctx = capi.Context(case.mesh, P2D, case.free, prec, m_max=M2D)
        for _ in range(3):
            ctx.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_LOCAL_CFL, CFL2D, M2D, info=False)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        for s in range(steps):
            flush.zero_()
            evs[s][0].record()
            ctx.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_LOCAL_CFL, CFL2D, M2D, info=False)
            evs[s][1].record()
        torch.cuda.synchronize()
        ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), dist)
        ctx.profile_enable(True)
        info = ctx.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_LOCAL_CFL, CFL2D, M2D)
        prof = ctx.profile_read()
        ctx.profile_enable(False)
        gs = second_pass_columns(list(info["reorth_cols"]), M2D)
        T = 8 if name == "fp64" else 4
        res[name] = {"value": ctx.K * steps / (ms / 1e3), "ms_per_step": ms / steps,
                     "kernel_ms_per_step": {k: round(v[1], 4) for k, v in prof.items() if v[0]},
                     "roofline": roofline_entry(prof, T, ctx.K, E, F, hbm, peak_kind, 2, P2D, M2D, "bump2d", fp64,
                                                fp32=fp32, gs=gs),
                     "second_pass_ran": round(gs[0], 4)}
        ctx.close()
    res["fp32_mixed"]["speedup_vs_fp64"] = res["fp64"]["ms_per_step"] / res["fp32_mixed"]["ms_per_step"]
    return {"workload": f"bump2d_{NX}x{NY}_p{P2D}_m{M2D}_pcexp_localcfl100", "steps": steps, **res}


def reference_arm(args, rank, world):
    """The oracle, as it stands, on the host cores: each step one PCEXP step of the same
    configuration (vortex, P2, m = 30, CFL 10) on a bounded sample (REF_SAMPLE_N^3 cubes)."""
    if rank != 0:
        return
    r = run_oracle(REF_SAMPLE_N, steps=args.steps, warm=args.warmup)
    total = sum(r["times"])
    value = r["K"] * args.steps / total
    sample = (f"{args.steps} PCEXP steps (after {args.warmup} untimed) of the same configuration on "
              f"{REF_SAMPLE_N}^3 cubes = {r['E']} tetrahedra (K = {r['K']}), FP64 numpy oracle, 1 thread "
              f"of {os.cpu_count()}")
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": WORKLOAD, "p": P3D, "m": M3D, "scheme": "PCEXP", "time_step": "global, CFL 10",
                   "sample": f"{REF_SAMPLE_N}^3 cubes, K={r['K']}"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "nproc": os.cpu_count(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


if __name__ == "__main__":
    main()
