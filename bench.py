#!/usr/bin/env python3
"""Throughput of the PCEXP Krylov step on GB300: DOF * steps / s.

Workload (default): the subsonic bump channel, 192 x 64 quads split into
24,576 triangles with +-15% node jitter (seed 1), DG P2 (K = 589,824
unknowns), Ma 0.5, slip walls and far-field boundaries, PCEXP with local time
steps at CFL 100 and Krylov dimension m = 30, FP64, starting from the free
stream.  One step = one PCEXP iteration (residual, two CGS2 Arnoldi
processes of 30 columns with their J v products, two phi evaluations, the
corrector residual and J v, both updates).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
For N > 1 run under torchrun; every rank runs an independent replica (the
path is not sharded), so the scaling is weak.
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
NX, NY, P, M, CFL, SEED = 192, 64, 2, 30, 100.0, 1
WORKLOAD = "bump2d_192x64_p2_m30_pcexp_localcfl100"
# bounded CPU samples of the same configuration (a smaller instance of the same channel)
CPU_SAMPLE = (96, 32)
REF_SAMPLE = (48, 16)


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
case = W.case_bump2d({nx}, {ny}, {p}, {seed})
dg = DGOracle(case.mesh, case.p, case.free)
u = np.zeros((dg.E, dg.nv, dg.N))
u[:, :, 0] = dg.freestream_state()[None, :] * np.sqrt(dg.area)[:, None]
u = u.reshape(-1)
times = []
for s in range({warm} + {steps}):
    t0 = time.perf_counter()
    u, _ = pcexp.steady_step(dg, u, {cfl}, {m})
    times.append(time.perf_counter() - t0)
print(json.dumps(dict(K=dg.K, times=times[{warm}:])))
"""


def run_oracle(nx, ny, steps, warm):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ORACLE_SNIPPET.format(root=ROOT, nx=nx, ny=ny, p=P, seed=SEED, warm=warm, steps=steps, cfl=CFL, m=M)
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
    return (p + 1) * (p + 2) * (p + 3) // 6, (p + 1) ** 3, (p + 1) ** 2, 5, 4


def algorithmic_bytes(kind, T, K, E, F, dim, p, m):
    """Minimum DRAM bytes per launch of a kernel class (per-kernel table of the design notes)."""
    nb, nq, nfq, nv, nf = shape(dim, p)
    geo = dim * dim + 2
    g_face = F * ((dim + 1) * T + 12)  # normal, measure, element and local-face ids
    g_elem = E * (geo * T + 4 * nf)    # inverse map, sqrt(det), h; face slots
    G = F * nfq * nv * T               # face-flux buffer
    avg_j = (m - 1) / 2.0              # mean column index over one Arnoldi process
    # J v element kernel: FP64 applies the volume point Jacobians (read v and the blocks,
    # write Jv); FP32-mixed recomputes the flux tangents at u_n (read u_n and v, write Jv)
    jvp_elem = (2 * K * T + dim * nv * nv * E * nq * T + E * (T + 4 * nf) + G if T == 8
                else 3 * K * T + g_elem + G)
    return {
        # face J v from the face point Jacobians: read v and the blocks, write G
        "jvp_face": K * T + 2 * nv * nv * F * nfq * T + F * 12 + G,
        "jvp_elem": jvp_elem,
        "residual_face": K * T + g_face + G,
        "residual_elem": 2 * K * T + g_elem + G,
        "cgs_proj": (avg_j + 2) * K * T,
        "cgs_upd_proj": (avg_j + 3) * K * T,
        "cgs_upd_norm": (avg_j + 3) * K * T,
    }.get(kind)


FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12  # SMs x DFMA/clk/SM x 2 flops x max SM clock

# DRAM bytes (read + write) per launch from one ncu capture of the same kernel on the same
# workload, keyed (workload, element bytes, kernel class); an entry is dropped when its
# kernel changes.  The summaries under profiles/ give the commands.
NCU_TRAFFIC = {
    ("bump2d", 8, "jvp_elem"): (67_718_656, "profiles/elem_apply_fp64_bump2d_p2.md"),
}


def algorithmic_flops(kind, K, E, F, dim, p, m):
    """Floating-point operations per launch of a kernel class (an FMA counts 2).

    jvp_elem: per element, nq points x (trace nv nb + Jacobian d nv^2) FMA and nv nb outputs x
    (volume d nq + lift nf nfq) FMA; jvp_face: per face point 2 nv nb trace + 2 nv^2 FMA;
    CGS kernels: per unknown and column, 1 (projection) or 2 (update + projection) FMA,
    averaged over the columns of one Arnoldi process."""
    nb, nq, nfq, nv, nf = shape(dim, p)
    nc = (m + 1) / 2.0  # mean number of basis columns per launch
    fma = {
        "jvp_elem": E * (nq * (nv * nb + dim * nv * nv) + nv * nb * (dim * nq + nf * nfq)),
        "jvp_face": F * nfq * (2 * nv * nb + 2 * nv * nv),
        "cgs_proj": K * (nc + 1),
        "cgs_upd_proj": K * 2 * nc,
        "cgs_upd_norm": K * (nc + 1),
    }.get(kind)
    return None if fma is None else 2.0 * fma


def roofline_entry(prof, precision_bytes, K, E, F, hbm, peak_kind, dim=2, p=2, m=30, workload="bump2d"):
    """Roofline of the dominant kernel class: FP64 kernels are bound by the FP64 pipe
    (alu, TFLOP/s), FP32 kernels by HBM (GB/s)."""
    dom = max(prof, key=lambda k: prof[k][1])
    n_dom, ms_dom = prof[dom]
    if not n_dom:
        return None
    sec = ms_dom / n_dom / 1e3
    tr = NCU_TRAFFIC.get((workload, precision_bytes, dom))
    entry = {"kernel": dom, "avg_launch_us": round(sec * 1e6, 2),
             "time_share": round(ms_dom / sum(v[1] for v in prof.values()), 4),
             "traffic": tr[0] if tr else None}
    if tr:
        entry["traffic_source"] = tr[1]
    ab = algorithmic_bytes(dom, precision_bytes, K, E, F, dim, p, m)
    if ab is not None:
        entry["algorithmic_bytes_per_launch"] = ab
    fl = algorithmic_flops(dom, K, E, F, dim, p, m)
    if precision_bytes == 8 and fl is not None:
        ach = fl / sec / 1e12
        entry.update({"bound": "alu", "achieved": round(ach, 3), "peak": round(FP64_PEAK_TFLOPS, 3),
                      "unit": "TFLOP/s", "frac": round(ach / FP64_PEAK_TFLOPS, 4),
                      "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 x 2.07 GHz",
                      "algorithmic_flops_per_launch": fl,
                      "hbm_frac": round(ab / sec / 1e9 / hbm, 4) if ab else None})
    elif ab is not None:
        ach = ab / sec / 1e9
        entry.update({"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                      "frac": round(ach / hbm, 4), "peak_source": peak_kind})
    return entry


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


def kernel_table(prof, precision_bytes, K, E, F, hbm, dim=2, p=2, m=30):
    """Every kernel class with a byte model: launches, mean launch time (CUDA events per
    class over the profiled steps), algorithmic GB/s and its fraction of measured HBM; FP64
    classes with a flop model also give TFLOP/s and the fraction of the FP64 pipe."""
    out = {}
    for kind, (n, ms) in prof.items():
        ab = algorithmic_bytes(kind, precision_bytes, K, E, F, dim, p, m)
        if not n or ab is None:
            continue
        sec = ms / n / 1e3
        row = {"launches": n, "avg_launch_us": round(sec * 1e6, 2), "gbs": round(ab / sec / 1e9, 1),
               "hbm_frac": round(ab / sec / 1e9 / hbm, 4)}
        fl = algorithmic_flops(kind, K, E, F, dim, p, m)
        if precision_bytes == 8 and fl is not None:
            row["fp64_tflops"] = round(fl / sec / 1e12, 3)
            row["fp64_frac"] = round(fl / sec / 1e12 / FP64_PEAK_TFLOPS, 4)
        out[kind] = row
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the second precision form")
    ap.add_argument("--no-3d", action="store_true", help="skip the 3D vortex block")
    ap.add_argument("--only-3d", action="store_true",
                    help="run the 3D vortex block alone and print it (profiling runs)")
    ap.add_argument("--n3d", type=int, default=48, help="cubes per side of the 3D vortex block")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"],
                    help="form of the headline value (the other form is reported beside it)")
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

    if args.only_3d:
        hbm, peak_kind = load_peaks()
        v3d = vortex3d_block(args, capi, W, torch, np, local, hbm, peak_kind, dist, world)
        if rank == 0:
            print(json.dumps({"vortex3d": v3d}))
        return

    case = W.case_bump2d(NX, NY, P, SEED)
    free = case.free
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def timed_steps(ctx, profile):
        """K steps after a barrier and a synchronize, L2 flushed before each step outside
        the step's CUDA events (recorded on the context's stream = torch's current stream)."""
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        if profile:
            ctx.profile_enable(True)
        for s in range(args.steps):
            flush.zero_()
            evs[s][0].record()
            ctx.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_LOCAL_CFL, CFL, M, info=False)
            evs[s][1].record()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ms = sum(a.elapsed_time(b) for a, b in evs)
        prof = ctx.profile_read() if profile else None
        if profile:
            ctx.profile_enable(False)
        return ms, prof

    def run(precision):
        ctx = capi.Context(case.mesh, P, free, precision, m_max=M)
        for _ in range(args.warmup):
            ctx.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_LOCAL_CFL, CFL, M, info=False)
        torch.cuda.synchronize()
        sampler = ClockSampler(local)
        sampler.start()
        ms, _ = timed_steps(ctx, False)          # the measurement
        ms_prof, prof = timed_steps(ctx, True)   # per-kernel-class events (adds launch gaps)
        clocks = sampler.stop()
        state = ctx.get_state()
        return ctx, ms, ms_prof, prof, clocks, state

    main_prec = capi.PCEXP_FP64 if args.precision == "fp64" else capi.PCEXP_FP32_MIXED
    ctx64, ms64, ms64_prof, prof, clocks, state64 = run(main_prec)
    K = ctx64.K
    ms_max = max_over_ranks(ms64, dist)
    value = job_throughput(K, args.steps, world, ms_max / 1e3)

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    hin = torch.empty(K, dtype=torch.float64, pin_memory=True).numpy()
    hout = torch.empty(K, dtype=torch.float64, pin_memory=True).numpy()
    ctx64.get_state(hin)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for s in range(args.steps):
        ctx64.set_state(hin)
        ctx64.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_LOCAL_CFL, CFL, M, info=False)
        ctx64.get_state(hout)
        hin, hout = hout, hin
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist)
    e2e_value = job_throughput(K, args.steps, world, e2e_s)

    # FP32-mixed form on the same workload.  Accuracy: one step from the same state in
    # both forms (the steady march at CFL 100 amplifies any 1e-7 difference to 1e-2
    # within a few steps, so multi-step state differences measure that, not FP32).
    mixed = None
    if not args.no_mixed and args.precision == "fp64":
        ctx32, ms32, ms32_prof, prof32, _, state32 = run(capi.PCEXP_FP32_MIXED)
        s0 = np.ascontiguousarray(state64)
        ctx64.set_state(s0)
        ctx64.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_LOCAL_CFL, CFL, M, info=False)
        a = ctx64.get_state()
        ctx32.set_state(s0)
        ctx32.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_LOCAL_CFL, CFL, M, info=False)
        b = ctx32.get_state()
        ms32 = max_over_ranks(ms32, dist)
        mixed = {"value": job_throughput(K, args.steps, world, ms32 / 1e3), "ms_per_step": ms32 / args.steps,
                 "speedup_vs_fp64": ms_max / ms32,
                 "one_step_state_rel_l2_vs_fp64": float(np.linalg.norm(b - a) / np.linalg.norm(a)),
                 "one_step_increment_rel_l2_vs_fp64": float(np.linalg.norm((b - s0) - (a - s0)) / np.linalg.norm(a - s0)),
                 "kernel_ms_per_step": {k: round(v[1] / args.steps, 4) for k, v in prof32.items() if v[0]}}
        ctx32.close()

    # roofline of the dominant kernel class (by device time in the timed region)
    hbm, peak_kind = load_peaks()
    E, nfq = case.mesh.n_elem, P + 1
    F = (3 * E + len(case.mesh.btags)) // 2
    launches = sum(v[0] for v in prof.values())
    Tb = 8 if args.precision == "fp64" else 4
    roof = roofline_entry(prof, Tb, K, E, F, hbm, peak_kind, 2, P, M)
    kernels = kernel_table(prof, Tb, K, E, F, hbm, 2, P, M)
    if mixed is not None:
        mixed["roofline"] = roofline_entry(prof32, 4, K, E, F, hbm, peak_kind, 2, P, M)
        mixed["kernels"] = kernel_table(prof32, 4, K, E, F, hbm, 2, P, M)
    ctx64.close()

    # the 3D vortex (48^3 cubes as 663,552 Kuhn tetrahedra, P2, K = 33,177,600), both forms
    v3d = None
    if not args.no_3d:
        v3d = vortex3d_block(args, capi, W, torch, np, local, hbm, peak_kind, dist, world)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = run_oracle(*CPU_SAMPLE, steps=1, warm=0)
        cpu = {"value": r["K"] * len(r["times"]) / sum(r["times"]), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"1 PCEXP local-step iteration of the same configuration on the "
                         f"{CPU_SAMPLE[0]}x{CPU_SAMPLE[1]} channel (K={r['K']}), FP64 numpy, 1 thread, "
                         f"{sum(r['times']):.1f} s"}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "mesh": f"{NX}x{NY} split quads, {E} triangles, 15% jitter seed {SEED}",
                   "p": P, "m": M, "K": K, "scheme": "PCEXP", "time_step": f"local, CFL {CFL:g}",
                   "precision": "FP64" if args.precision == "fp64" else "FP32-mixed", "l2": "flushed between steps (256 MB write outside the step events)",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": K * 8, "d2h_bytes_per_step": K * 8},
        "gpu_launches": launches,
        "ms_per_step_with_kernel_events": ms64_prof / args.steps,
        "kernel_ms_per_step": {k: round(v[1] / args.steps, 4) for k, v in prof.items() if v[0]},
        "roofline": roof,
        "kernels": kernels,
        "kernels_note": ("algorithmic bytes (and FP64 flops) per launch over CUDA-event time per kernel "
                         "class; at this size a Krylov basis of 31 vectors (146 MB FP64, 73 MB FP32) is "
                         "partly or wholly L2-resident, so Gram-Schmidt fractions of HBM can exceed 1"),
        "cpu_baseline": cpu,
        "fp32_mixed": mixed,
        "vortex3d": v3d,
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def vortex3d_block(args, capi, W, torch, np, local, hbm, peak_kind, dist=None, world=1):
    """Throughput of PCEXP steps on the 3D vortex (global CFL 10, m = 30) in both forms from
    the projected vortex, with CUDA events per step after warm-up (inputs far larger than
    L2), the dominant kernel's roofline and the FP32-mixed state error against FP64 after
    the same steps."""
    case = W.case_vortex3d(n=args.n3d)
    steps, warm = max(3, min(args.steps, 5)), 3
    prm = [case.vortex.eps, *case.vortex.center, 10.0]
    res, states = {}, {}
    for name, prec in (("fp64", capi.PCEXP_FP64), ("fp32_mixed", capi.PCEXP_FP32_MIXED)):
        ctx = capi.Context(case.mesh, case.p, case.free, prec, m_max=case.m)
        ctx.project_state(capi.PCEXP_PROJ_VORTEX, prm)
        for _ in range(warm):
            ctx.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GLOBAL_CFL, case.cfl, case.m, info=False)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        for s in range(steps):
            evs[s][0].record()
            ctx.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GLOBAL_CFL, case.cfl, case.m, info=False)
            evs[s][1].record()
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in evs)
        ctx.profile_enable(True)
        ctx.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GLOBAL_CFL, case.cfl, case.m, info=False)
        torch.cuda.synchronize()
        prof = ctx.profile_read()
        ctx.profile_enable(False)
        K, E = ctx.K, case.mesh.n_elem
        F = 2 * E  # periodic: every face interior
        states[name] = ctx.get_state()
        ms = max_over_ranks(ms, dist)
        res[name] = {"value": job_throughput(K, steps, world, ms / 1e3), "ms_per_step": ms / steps,
                     "kernel_ms_per_step": {k: round(v[1], 3) for k, v in prof.items() if v[0]},
                     "roofline": roofline_entry(prof, 8 if name == "fp64" else 4, K, E, F, hbm, peak_kind,
                                                3, case.p, case.m, "vortex3d"),
                     "kernels": kernel_table(prof, 8 if name == "fp64" else 4, K, E, F, hbm, 3, case.p, case.m)}
        ctx.close()
    a, b = states["fp64"], states["fp32_mixed"]
    res["fp32_mixed"]["speedup_vs_fp64"] = res["fp64"]["ms_per_step"] / res["fp32_mixed"]["ms_per_step"]
    res["fp32_mixed"]["state_rel_l2_vs_fp64"] = float(np.linalg.norm(b - a) / np.linalg.norm(a))
    n = args.n3d
    return {"workload": f"vortex3d_{n}cubed_p2_m30_pcexp_globalcfl10",
            "mesh": f"{n}^3 cubes, {6 * n ** 3:,} Kuhn tetrahedra, 10% jitter seed 5, periodic [0,10]^3",
            "K": K, "steps": steps, "warmup": warm,
            "note": f"state error after {warm + steps} steps from the projected vortex in both forms",
            **res}


def reference_arm(args, rank, world):
    """The oracle, as it stands, on the host cores: each step one PCEXP iteration on a
    bounded sample (the same channel configuration at REF_SAMPLE resolution)."""
    if rank != 0:
        return
    r = run_oracle(*REF_SAMPLE, steps=args.steps, warm=args.warmup)
    total = sum(r["times"])
    value = r["K"] * args.steps / total
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": WORKLOAD, "p": P, "m": M, "scheme": "PCEXP", "time_step": f"local, CFL {CFL:g}",
                   "sample": f"{REF_SAMPLE[0]}x{REF_SAMPLE[1]} channel, K={r['K']}"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} PCEXP local-step iterations of the same configuration on the "
                                   f"{REF_SAMPLE[0]}x{REF_SAMPLE[1]} channel (K={r['K']}), FP64 numpy, 1 thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


if __name__ == "__main__":
    main()
