"""Benchmark of the LOPe stencil hot path on GB300.

One step = the plain method at scale: 3D 7-point diffusion (FP32, 512^3,
Dirichlet 0, c = 0.1, 50 sweeps) followed by the 2D 9-point radius-2 star
(FP32, 8192^2, periodic, c = 0.1, 50 sweeps), both through lope_apply with
their inputs resident in HBM.  `value` is grid-point updates per second over
the whole job.  Each buffer (512 MiB, 256 MiB) is larger than L2, so no L2
flush is needed between steps.

Extra forms (outside the timed region, reported under "forms"): the batched
launch (512 uneven 2D grids, 20 steps) against per-grid launches, the forward +
adjoint (256^3, 100 steps, checkpoint every 10) against the plain forward,
the shallow-water multi-field forms (linear, and nonlinear flux form with a box
halo) in FP32 and BF16, SSP-RK3 steps of the nonlinear form (fused against one
launch per stage), local functions written as source and compiled at run time
(against the builtin, and Gray-Scott), and the FP64 256^2 case.

--impl reference times the FP64 oracle on the host cores instead (bounded
samples of the same workload mix).  Under torchrun every rank runs its own
replica (the grids are independent problems; no collective is on the path).
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
sys.path.insert(0, ROOT)

METRIC = "grid-point updates/s and HBM GB/s vs peak; batched and fwd+adjoint vs plain"
UNIT = "grid-point updates/s"
N3, T3, C3 = 512, 50, 0.1
N2, T2, C2 = 8192, 50, 0.1
UPD3 = N3 ** 3 * T3
UPD2 = N2 ** 2 * T2
WORKLOAD = ("3D 7-point diffusion FP32 512^3 Dirichlet-0 c=0.1 x50 sweeps + "
            "2D 9-point r=2 star FP32 8192^2 periodic c=0.1 x50 sweeps")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def max_over_ranks(value, pg, device):
    """Largest value over all ranks (the job's wall time is its slowest rank)."""
    if pg is None:
        return value
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, out_dir=None):
        self.proc, self.path, self.gpu, self.out_dir = None, None, gpu_index, out_dir

    def start(self):
        try:
            # the samples go to --clocks-dir when given, else to a temporary file
            if self.out_dir:
                os.makedirs(self.out_dir, exist_ok=True)
                self.path = os.path.join(self.out_dir, f"clocks_rank{self.gpu}.csv")
            else:
                import tempfile
                fd, self.path = tempfile.mkstemp(prefix=f"lope_clocks_rank{self.gpu}_", suffix=".csv")
                os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx = max(mx, float(f[2]))
                except ValueError:
                    continue
                for n, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        if not self.out_dir:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- CPU baseline
def _full_inputs():
    """The benchmark step's two grids at full size, FP64 (the oracle's type)."""
    import lope_inputs as LI

    u3 = LI.uniform_field(1001, (N3, N3, N3)).astype(np.float32).astype(np.float64)
    u2 = LI.uniform_field(1001, (N2, N2), offset=1 << 32).astype(np.float32).astype(np.float64)
    return u3, u2


def oracle_rates(u3=None, u2=None):
    """Oracle point-updates/s on this host for the benchmark step: one timed
    sweep of each full-size grid (512^3 diff7, 8192^2 star9r2) on all cores
    and on one thread, extrapolated to the step's 50 + 50 sweeps."""
    import oracle

    oracle.build()
    th = oracle.max_threads()
    if u3 is None:
        u3, u2 = _full_inputs()
    t = {}
    for nth in (th, 1):
        t0 = time.perf_counter()
        oracle.apply(u3, "diff7", [C3], 1, bc=[1, 1, 1], nthreads=nth)
        t1 = time.perf_counter()
        oracle.apply(u2, "star9r2", [C2], 1, nthreads=nth)
        t[nth] = (t1 - t0, time.perf_counter() - t1)
    (a3, a2), (b3, b2) = t[th], t[1]
    return {"value": (UPD3 + UPD2) / (T3 * a3 + T2 * a2), "unit": UNIT, "cores": th,
            "kind": "oracle",
            "sample": f"one sweep of each full-size grid of the step (diff7 {N3}^3 Dirichlet 0: "
                      f"{a3:.2f} s, star9r2 {N2}^2 periodic: {a2:.2f} s; FP64 oracle, OpenMP "
                      f"{th} threads), extrapolated to the step's {T3} + {T2} sweeps",
            "value_1thread": (UPD3 + UPD2) / (T3 * b3 + T2 * b2),
            "sample_1thread": f"the same sweeps on one thread ({b3:.1f} s + {b2:.1f} s)",
            "same_config": True}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle

    oracle.build()
    th = oracle.max_threads()
    u3, u2 = _full_inputs()

    def step():  # one sweep of each full-size grid: the step's 2:1 update mix
        oracle.apply(u3, "diff7", [C3], 1, bc=[1, 1, 1], nthreads=th)
        oracle.apply(u2, "star9r2", [C2], 1, nthreads=th)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    upd = (u3.size + u2.size) * args.steps
    v = upd / dt
    sample = (f"per step: one sweep of diff7 {N3}^3 Dirichlet 0 and one of star9r2 {N2}^2 "
              f"periodic, the full-size grids of the GPU step with 1 of its {T3} + {T2} sweeps "
              f"(FP64 oracle, plain C loops, OpenMP {th} threads)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD + " (1 + 1 of the sweeps per step)"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": th, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------- GPU arm
KERNEL_SOURCES = ("k_tma.cu", "tma_kernels.cuh", "tma_device.cuh", "device_common.cuh",
                  "lope_internal.h")


def kernel_source_hash():
    """Hash of the sources the TMA kernels are compiled from."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1502_03504_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_record():
    """Per-launch DRAM bytes from the committed ncu summary, if it matches the source."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            rec = json.load(fh)
        if rec.get("source_sha256_16") == kernel_source_hash():
            return rec
    except Exception:
        pass
    return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lope", choices=["lope", "reference"])
    ap.add_argument("--main-only", action="store_true", help="skip the extra forms")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline")
    ap.add_argument("--clocks-dir", default=None,
                    help="keep the nvidia-smi clock samples of the timed region in this folder")
    ap.add_argument("--profile", default=None,
                    help="run one kernel workload for --steps launches and exit (for ncu): "
                         "diff7:N, diff7p:N, star9r2:N, jacobi5:N, swe:N, swebf16:N, sweflux:N, "
                         "swefluxbf16:N, with an optional boundary spec per axis, slowest first, "
                         "e.g. diff7:512:DDP (D Dirichlet 0, P periodic), and :k2 for two sweeps "
                         "per launch; batch:NGRIDS[:trap] for the first NGRIDS grids of the "
                         "batched workload")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile:
        return run_profile(args)

    import torch

    import lope_inputs as LI
    import paper_1502_03504_gb300 as L
    from paper_1502_03504_gb300 import build as B

    ws, rank, local = dist_env()
    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    def barrier():
        if pg:
            pg.barrier()
        torch.cuda.synchronize()

    # ---------------- inputs (seeded, on the host, then resident in HBM)
    u3_h = torch.from_numpy(LI.uniform_field(1001, (N3, N3, N3)).astype(np.float32)).pin_memory()
    u2_h = torch.from_numpy(LI.uniform_field(1001, (N2, N2), offset=1 << 32).astype(np.float32)).pin_memory()
    u3 = u3_h.to(dev)
    u2 = u2_h.to(dev)
    o3, w3 = torch.empty_like(u3), torch.empty_like(u3)
    o2, w2 = torch.empty_like(u2), torch.empty_like(u2)
    g3 = L.Grid((N3, N3, N3), "f32", halo=1).set_boundary(kind="dirichlet", value=0.0)
    s3 = L.Stencil.builtin("diff7", C3)
    g2 = L.Grid((N2, N2), "f32", halo=2)
    s2 = L.Stencil.builtin("star9r2", C2)
    stream = torch.cuda.current_stream(dev)

    def step():
        L.apply(g3, s3, u3, out=o3, work=w3, nsteps=T3)
        L.apply(g2, s2, u2, out=o2, work=w2, nsteps=T2)

    for _ in range(max(3, args.warmup)):
        step()
    L.sync_status()

    # ---------------- timed region: device-resident inputs
    clocks = Clocks(local, args.clocks_dir)
    clocks.start()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    n0 = L.launch_count()
    start.record(stream)
    for i in range(args.steps):
        ev[i][0].record(stream)
        L.apply(g3, s3, u3, out=o3, work=w3, nsteps=T3)
        ev[i][1].record(stream)
        L.apply(g2, s2, u2, out=o2, work=w2, nsteps=T2)
        ev[i][2].record(stream)
    end.record(stream)
    barrier()
    launches = L.launch_count() - n0
    clk = clocks.stop()
    L.sync_status()
    ms = start.elapsed_time(end)
    t3 = sum(e[0].elapsed_time(e[1]) for e in ev) / args.steps
    t2 = sum(e[1].elapsed_time(e[2]) for e in ev) / args.steps
    ms = max_over_ranks(ms, pg, dev)
    upd_step = UPD3 + UPD2
    value = upd_step * args.steps * ws / (ms / 1e3)

    # ---------------- end to end: host buffers, copies inside the timed region.
    # Every step goes through lope_apply_host (host -> device copy, the sweeps,
    # device -> host copy of the result) for each grid.  Consecutive steps
    # alternate between two streams and two device-buffer sets per grid, so one
    # step's copies overlap another step's sweeps, as a pipeline of batches.
    nset = 2
    h_o3 = [torch.empty_like(u3_h).pin_memory() for _ in range(nset)]
    h_o2 = [torch.empty_like(u2_h).pin_memory() for _ in range(nset)]
    d3 = [(u3, o3, w3)] + [tuple(torch.empty_like(u3) for _ in range(3)) for _ in range(nset - 1)]
    d2 = [(u2, o2, w2)] + [tuple(torch.empty_like(u2) for _ in range(3)) for _ in range(nset - 1)]
    sts = [torch.cuda.Stream(dev) for _ in range(nset)]
    e2e_steps = max(4, args.steps // 2)

    def e2e_step(i):
        k = i % nset
        L.apply_host(g3, s3, u3_h, h_o3[k], d3[k][0], d3[k][1], d3[k][2], nsteps=T3, stream=sts[k])
        L.apply_host(g2, s2, u2_h, h_o2[k], d2[k][0], d2[k][1], d2[k][2], nsteps=T2, stream=sts[k])

    e2e_step(0)  # warm-up of the host-buffer path
    e2e_step(1)
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for st_ in sts:
        st_.wait_event(e0)
    for i in range(e2e_steps):
        e2e_step(i)
    for st_ in sts:
        stream.wait_stream(st_)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), pg, dev)
    # The same steps without the pipeline: all on one stream, so every copy
    # waits for the sweeps before it.
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    sts[0].wait_event(s0)
    for _ in range(e2e_steps):
        e2e_step(0)
    stream.wait_stream(sts[0])
    s1.record(stream)
    torch.cuda.synchronize()
    serial_ms = max_over_ranks(s0.elapsed_time(s1), pg, dev)
    e2e = {"value": upd_step * e2e_steps * ws / (e2e_ms / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": u3.numel() * 4 + u2.numel() * 4,
           "d2h_bytes_per_step": o3.numel() * 4 + o2.numel() * 4,
           "api": "lope_apply_host per grid (pinned host buffers); consecutive steps alternate "
                  "between 2 streams and 2 device-buffer sets, so one step's copies overlap "
                  "the other's sweeps",
           "steps": e2e_steps,
           "unpipelined_value": upd_step * e2e_steps * ws / (serial_ms / 1e3)}
    del d3, d2

    # ---------------- roofline of the dominant kernel (3D TMA z-march)
    # The plan of each grid (path, temporal depth k, launches) comes from the
    # library.  One launch reads each point once and writes it once (8 B per
    # FP32 point) while it advances k sweeps, so its algorithmic bytes are
    # 8 B x points and an update costs 8/k B; "effective" counts 8 B per update.
    peak, peak_kind = peaks()
    plan3, nl3 = L.plan(g3, s3, u3, o3, w3, nsteps=T3)
    plan2, nl2 = L.plan(g2, s2, u2, o2, w2, nsteps=T2)
    k3, k2 = plan3.tsteps, plan2.tsteps
    alg3 = 8.0 * N3 ** 3
    alg2 = 8.0 * N2 ** 2
    launch3_s = t3 / 1e3 / nl3
    launch2_s = t2 / 1e3 / nl2
    ach3 = alg3 / launch3_s / 1e9
    ach2 = alg2 / launch2_s / 1e9
    tr = traffic_record()
    name3 = ("tma3d_tb2s_kernel<OpDiff7, float> (512^3, two sweeps per launch)" if k3 == 2 else
             "tma3d_kernel<OpDiff7, float> (512^3, one sweep per launch)")
    roofline = {"bound": "hbm", "achieved": ach3, "peak": peak, "unit": "GB/s",
                "frac": ach3 / peak,
                "traffic": tr.get(f"diff7_512_k{k3}_bytes_per_launch") if tr else None,
                "kernel": name3, "sweeps_per_launch": k3,
                "alg_bytes_per_launch": alg3, "avg_launch_us": launch3_s * 1e6,
                "effective_GBps": ach3 * k3, "effective_frac": ach3 * k3 / peak,
                "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})"}
    kernels = {
        "diff7_512": {"share_of_step": t3 / (t3 + t2), "sweeps_per_launch": k3, "launches": nl3,
                      "avg_launch_us": launch3_s * 1e6, "alg_GBps": ach3, "frac_of_peak": ach3 / peak,
                      "updates_per_s": N3 ** 3 * T3 / (t3 / 1e3)},
        "star9r2_8192": {"share_of_step": t2 / (t3 + t2), "sweeps_per_launch": k2, "launches": nl2,
                         "avg_launch_us": launch2_s * 1e6,
                         "alg_GBps": ach2, "frac_of_peak": ach2 / peak,
                         "updates_per_s": N2 ** 2 * T2 / (t2 / 1e3),
                         "traffic": tr.get(f"star9r2_8192_k{k2}_bytes_per_launch") if tr else None},
    }
    # the one-sweep z-march on the same grid (the k = 1 form of the roofline
    # gate), timed after the step
    one = L.Launch(1, 0, 0, 1, -1)
    L.apply(g3, s3, u3, out=o3, work=w3, nsteps=T3, launch=one)
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    L.apply(g3, s3, u3, out=o3, work=w3, nsteps=T3, launch=one)
    g1.record(stream)
    torch.cuda.synchronize()
    k1_s = g0.elapsed_time(g1) / 1e3 / T3
    kernels["diff7_512_one_sweep_per_launch"] = {
        "avg_launch_us": k1_s * 1e6, "alg_GBps": alg3 / k1_s / 1e9,
        "frac_of_peak": alg3 / k1_s / 1e9 / peak, "updates_per_s": N3 ** 3 / k1_s,
        "traffic": tr.get("diff7_512_k1_bytes_per_launch") if tr else None}

    forms = {}
    if not args.main_only and rank == 0:
        del u3_h, u2_h, h_o3, h_o2
        for name, fn in (("fp64_256", form_fp64), ("swe_4096", form_swe), ("batched_512", form_batch),
                         ("fwd_adjoint_256", form_adjoint), ("swe_flux_4096", form_swe_flux),
                         ("rk3_swe_flux_4096", form_rk3), ("user_source", form_user_source)):
            try:
                forms[name] = fn(L, LI, torch, dev, peak)
            except Exception as e:  # reported, never hidden
                forms[name] = {"error": f"{type(e).__name__}: {e}"}
            torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = oracle_rates()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "updates_per_step": upd_step,
                       "parallelism": f"replicas{ws}" if ws > 1 else "single",
                       "l2": "inputs larger than L2 (512 MiB and 256 MiB per buffer); no flush",
                       "launch": f"lope_apply auto plan: TMA z-march (3D, {k3} sweeps per launch), "
                                 f"TMA tiles (2D, {k2} sweep per launch)"},
            "e2e": e2e, "gpu_launches": launches, "clocks": clk, "roofline": roofline,
            "kernels": kernels, "cpu_baseline": cpu, "forms": forms,
        }
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


# ---------------------------------------------------------------- profiling cases
def run_profile(args):
    """One workload, --warmup + --steps single-sweep launches; prints per-launch time."""
    import torch

    import lope_inputs as LI
    import paper_1502_03504_gb300 as L
    from paper_1502_03504_gb300 import build as B

    B.build()
    parts = args.profile.split(":")
    ksw = 2 if "k2" in parts[2:] else 1  # sweeps per launch (the two-sweep z-march)
    parts = [q for q in parts if q != "k2"]
    name = parts[0]
    dims = [int(x) for x in parts[1].split("x")]
    n = dims[0]
    spec = parts[2] if len(parts) > 2 else None
    dev = torch.device("cuda", 0)
    if name in ("diff7", "diff7p", "diff7bf16"):
        shape = tuple(dims) if len(dims) == 3 else (n, n, n)
        st, halo, pts = L.Stencil.builtin("diff7", C3), 1, int(np.prod(shape))
        kind, nf = ("periodic" if name == "diff7p" else "dirichlet"), 1
        dtype, bpp = ("bf16", 4) if name == "diff7bf16" else ("f32", 8)
    elif name in ("star9r2", "jacobi5"):
        shape = tuple(dims) if len(dims) == 2 else (n, n)
        halo, pts = 2 if name == "star9r2" else 1, int(np.prod(shape))
        st = L.Stencil.builtin(name, 0.1 if name == "star9r2" else 0.2)
        kind, nf, dtype, bpp = "periodic", 1, "f32", 8
    elif name in ("swe", "swebf16"):
        shape, halo, pts = (n, n), 1, n * n
        st = L.Stencil.builtin("swe_cgrid", 0.02, 1.0, 1.0)
        kind, nf = "periodic", 3
        dtype, bpp = ("f32", 24) if name == "swe" else ("bf16", 12)
    elif name == "batch":
        return run_profile_batch(args, n, trap="trap" in parts[2:])
    elif name in ("sweflux", "swefluxbf16"):
        shape, halo, pts = (n, n), 1, n * n
        st = L.Stencil.builtin("swe_flux", 0.02, 1.0, 0.5, 1.0)
        kind, nf = "periodic", 3
        dtype, bpp = ("f32", 24) if name == "sweflux" else ("bf16", 12)
    else:
        raise SystemExit(f"unknown profile case {name}")
    g = L.Grid(shape, dtype, halo=halo, nfields=nf)
    if spec:
        g.set_boundaries([0 if c == "P" else 1 for c in spec])
    elif kind == "dirichlet":
        g.set_boundary(kind="dirichlet", value=0.0)
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16}[dtype]
    fields = [torch.from_numpy(LI.uniform(1001, pts, k * pts).astype(np.float32).reshape(shape))
              .to(dev).to(tdt) for k in range(nf)]
    outs = [torch.empty_like(f) for f in fields]
    works = [torch.empty_like(f) for f in fields]
    launch = L.Launch(1, 0, 0, ksw, -1) if ksw == 2 else None
    for _ in range(args.warmup):
        L.apply(g, st, fields, out=outs, work=works, nsteps=ksw, launch=launch)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        L.apply(g, st, fields, out=outs, work=works, nsteps=ksw, launch=launch)
    b.record()
    torch.cuda.synchronize()
    L.sync_status()
    us = a.elapsed_time(b) / args.steps * 1e3
    print(json.dumps({"profile": args.profile, "us_per_launch": us,
                      "alg_GBps": bpp * pts / (us * 1e-6) / 1e9}), flush=True)


def run_profile_batch(args, ngrids, trap=False):
    """The first `ngrids` grids of the batched workload: one batched launch per
    step of 4 sweeps; the planner's default (two-sweep tiles, two passes) or,
    with `trap`, the trapezoid tiles (128 x 32, 4 sweeps = one pass)."""
    import torch

    import lope_inputs as LI
    import paper_1502_03504_gb300 as L

    dev = torch.device("cuda", 0)
    shapes, kinds = LI.batch_shapes(1003, 512)
    shapes, kinds = shapes[:ngrids], kinds[:ngrids]
    grids, ins = [], []
    for (ny, nx), k in zip(shapes, kinds):
        g = L.Grid((ny, nx), "f32", halo=1)
        g.set_boundaries([k, k])
        grids.append(g)
        ins.append(torch.from_numpy(LI.uniform_field(1003, (ny, nx)).astype(np.float32)).to(dev))
    outs = [torch.empty_like(x) for x in ins]
    works = [torch.empty_like(x) for x in ins]
    s = L.Stencil.builtin("jacobi5", 0.2)
    cfg = L.Launch(2, 128, 32, 4, -1) if trap else None
    wsb = torch.empty(L.batch_workspace_size(grids, s), dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        L.apply_batch(grids, s, ins, outs, works, 4, cfg, wsb)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        L.apply_batch(grids, s, ins, outs, works, 4, cfg, wsb)
    b.record()
    torch.cuda.synchronize()
    L.sync_status()
    pts = sum(y * x for y, x in shapes)
    ms = a.elapsed_time(b) / args.steps
    print(json.dumps({"profile": f"batch:{ngrids}", "points": pts, "ms_per_launch": ms,
                      "updates_per_s": 4 * pts / (ms / 1e3)}), flush=True)


# ---------------------------------------------------------------- extra forms
def _time(torch, fn, reps=5):
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _sweeps_per_launch(L, g, s, f, o, w, T):
    """Temporal depth of the plan apply() runs (host only, no CUDA call).
    The forms' "effective" figures count every sweep's read and write of each
    field, as one sweep per launch moves them."""
    launch, _ = L.plan(g, s, f, o, w, nsteps=T)
    return max(1, launch.tsteps)


def form_fp64(L, LI, torch, dev, peak):
    u = torch.from_numpy(LI.uniform_field(1000, (256, 256))).to(dev)
    g = L.Grid((256, 256), "f64", halo=1)
    s = L.Stencil.builtin("jacobi5", 0.2)
    o, w = torch.empty_like(u), torch.empty_like(u)
    ms = _time(torch, lambda: L.apply(g, s, u, out=o, work=w, nsteps=100), reps=20)
    return {"workload": "jacobi5 FP64 256^2 periodic x100 (L2-resident, graph-replayed)",
            "ms": ms, "updates_per_s": 256 * 256 * 100 / (ms / 1e3)}


def form_swe(L, LI, torch, dev, peak):
    n, T = 4096, 200
    h, u, v = LI.swe_fields(1002, (n, n))
    res = {}
    for dtype, tdt, first in (("f32", torch.float32, h), ("bf16", torch.bfloat16, h - 1.0)):
        f = [torch.from_numpy(LI.to_storage(x, "bf16" if dtype == "bf16" else "f32")).to(dev).to(tdt)
             for x in (first, u, v)]
        o = [torch.empty_like(x) for x in f]
        w = [torch.empty_like(x) for x in f]
        g = L.Grid((n, n), dtype, halo=1, nfields=3)
        s = L.Stencil.builtin("swe_cgrid", 0.02, 1.0, 1.0)
        ms = _time(torch, lambda: L.apply(g, s, f, out=o, work=w, nsteps=T), reps=3)
        esz = 4 if dtype == "f32" else 2
        gbps = 6 * esz * n * n * T / (ms / 1e3) / 1e9
        res[dtype] = {"ms": ms, "point_updates_per_s": n * n * T / (ms / 1e3),
                      "sweeps_per_launch": _sweeps_per_launch(L, g, s, f, o, w, T),
                      "effective_GBps": gbps, "effective_frac": gbps / peak}
        del f, o, w
    res["bf16_speedup_vs_f32"] = res["f32"]["ms"] / res["bf16"]["ms"]
    res["workload"] = "C-grid shallow water (h,u,v) 4096^2 periodic x200; BF16 stores eta = h - 1"
    return res


def _flux_fields(LI, torch, dev, n, dtype, seed):
    h, u, v = LI.swe_fields(seed, (n, n))
    tdt = torch.float32 if dtype == "f32" else torch.bfloat16
    return [torch.from_numpy(LI.to_storage(x, dtype)).to(dev).to(tdt) for x in (h - 1.0, u, v)]


def form_swe_flux(L, LI, torch, dev, peak):
    """Nonlinear flux-form shallow water (box halo, corner taps), 4096^2 x 3
    fields, periodic, 200 forward-Euler steps, FP32 and BF16 storage."""
    n, T = 4096, 200
    res = {}
    for dtype in ("f32", "bf16"):
        f = _flux_fields(LI, torch, dev, n, dtype, 1009)
        o = [torch.empty_like(x) for x in f]
        w = [torch.empty_like(x) for x in f]
        g = L.Grid((n, n), dtype, halo=1, nfields=3)
        s = L.Stencil.builtin("swe_flux", 0.02, 1.0, 0.5, 1.0)
        ms = _time(torch, lambda: L.apply(g, s, f, out=o, work=w, nsteps=T), reps=3)
        esz = 4 if dtype == "f32" else 2
        gbps = 6 * esz * n * n * T / (ms / 1e3) / 1e9
        res[dtype] = {"ms": ms, "point_updates_per_s": n * n * T / (ms / 1e3),
                      "alg_GBps": gbps, "frac_of_peak": gbps / peak}
        del f, o, w
    res["bf16_speedup_vs_f32"] = res["f32"]["ms"] / res["bf16"]["ms"]
    res["workload"] = ("nonlinear flux-form C-grid shallow water (eta,u,v) 4096^2 periodic x200, "
                       "dt 0.02, g 1, f 0.5, H 1; TMA tiles with box halo")
    return res


def form_rk3(L, LI, torch, dev, peak):
    """SSP-RK3 steps of the nonlinear shallow water, 4096^2 x 3 FP32, 50 steps:
    fused trapezoid steps (stage states in shared memory) against one launch
    per stage (TMA tiles, stage states in HBM) and against 150 plain sweeps."""
    n, T = 4096, 50
    f = _flux_fields(LI, torch, dev, n, "f32", 1105)
    o = [torch.empty_like(x) for x in f]
    w = [torch.empty((2, n, n), dtype=x.dtype, device=dev) for x in f]
    g = L.Grid((n, n), "f32", halo=1, nfields=3)
    s = L.Stencil.builtin("swe_flux", 0.02, 1.0, 0.5, 1.0).set_scheme("rk3")
    best = None
    for tx, ty in ((64, 32), (64, 16), (128, 16), (32, 32)):
        for k in (1, 2):
            cfg = L.Launch(2, tx, ty, k, -1)
            try:
                ms = _time(torch, lambda: L.apply(g, s, f, out=o, work=w, nsteps=T, launch=cfg), reps=2)
            except Exception:
                continue
            if best is None or ms < best[0]:
                best = (ms, tx, ty, k)
    ms_fused, tx, ty, k = best
    ms_stage = _time(torch, lambda: L.apply(g, s, f, out=o, work=w, nsteps=T,
                                            launch=L.Launch(1, 0, 0, 0, -1)), reps=3)
    e = L.Stencil.builtin("swe_flux", 0.02, 1.0, 0.5, 1.0)
    ms_euler = _time(torch, lambda: L.apply(g, e, f, out=o, work=[x[0] for x in w], nsteps=3 * T), reps=3)
    pts = n * n * T
    return {"workload": "SSP-RK3 nonlinear shallow water 4096^2 x3 FP32 periodic x50 steps (150 stages)",
            "fused_trapezoid_ms": ms_fused, "fused_choice": {"tile": [tx, ty], "tsteps": k},
            "fused_rk_steps_per_s": pts / (ms_fused / 1e3),
            "fused_alg_GBps": 24 * pts / (ms_fused / 1e3) / 1e9,
            "fused_frac_of_peak": 24 * pts / (ms_fused / 1e3) / 1e9 / peak,
            "stage_launches_ms": ms_stage, "stage_alg_GBps": 96 * pts / (ms_stage / 1e3) / 1e9,
            "stage_frac_of_peak": 96 * pts / (ms_stage / 1e3) / 1e9 / peak,
            "euler_150_sweeps_ms": ms_euler,
            "fused_speedup_vs_stage_launches": ms_stage / ms_fused}


# Local functions written as source (compiled at run time by the library).
SRC_DIFF7 = """
const C u = U(0, 0, 0, 0);
const C nb = add(add(add(U(0, -1, 0, 0), U(0, 1, 0, 0)), add(U(0, 0, -1, 0), U(0, 0, 1, 0))),
                 add(U(0, 0, 0, -1), U(0, 0, 0, 1)));
out[0] = fma_(P[0], fma_(C(-6), u, nb), u);
"""
SRC_GRAY_SCOTT = """
const C u = U(0, 0, 0), v = U(1, 0, 0);
const C lu = fma_(C(-4), u, add(add(U(0, -1, 0), U(0, 1, 0)), add(U(0, 0, -1), U(0, 0, 1))));
const C lv = fma_(C(-4), v, add(add(U(1, -1, 0), U(1, 1, 0)), add(U(1, 0, -1), U(1, 0, 1))));
const C uvv = mul(u, mul(v, v));
out[0] = fma_(P[0], fma_(P[1], lu, fma_(P[3], sub(C(1), u), -uvv)), u);
out[1] = fma_(P[0], fma_(P[2], lv, fma_(-add(P[3], P[4]), v, uvv)), v);
"""


def form_user_source(L, LI, torch, dev, peak):
    """User-written local functions compiled at run time: the 3D 7-point
    diffusion written as source against the builtin (512^3 FP32 Dirichlet-0,
    50 sweeps), and Gray-Scott reaction-diffusion (two coupled nonlinear
    fields, no builtin) at 4096^2 FP32 periodic, 100 steps."""
    n3, T3 = 512, 50
    u = torch.from_numpy(LI.uniform_field(1001, (n3, n3, n3)).astype(np.float32)).to(dev)
    o, w = torch.empty_like(u), torch.empty_like(u)
    g = L.Grid((n3, n3, n3), "f32", halo=1)
    g.set_boundary(kind="dirichlet", value=0.0)
    src = L.Stencil.source(SRC_DIFF7, ndim=3, radius=1, params=[C3]).compile("f32")
    ms_src = _time(torch, lambda: L.apply(g, src, u, out=o, work=w, nsteps=T3), reps=3)
    ms_blt = _time(torch, lambda: L.apply(g, L.Stencil.builtin("diff7", C3), u, out=o, work=w,
                                          nsteps=T3), reps=3)
    del u, o, w
    n, T = 4096, 100
    prm = [1.0, 0.16, 0.08, 0.035, 0.065]
    f = [torch.from_numpy((1.0 - 0.3 * LI.uniform_field(1205, (n, n))).astype(np.float32)).to(dev),
         torch.from_numpy((0.25 * LI.uniform_field(1205, (n, n), offset=n * n)).astype(np.float32)).to(dev)]
    fo = [torch.empty_like(x) for x in f]
    fw = [torch.empty_like(x) for x in f]
    g2 = L.Grid((n, n), "f32", halo=1, nfields=2)
    gs = L.Stencil.source(SRC_GRAY_SCOTT, ndim=2, radius=1, nfields=2, params=prm).compile("f32")
    ms_gs = _time(torch, lambda: L.apply(g2, gs, f, out=fo, work=fw, nsteps=T), reps=3)
    gbps = 16 * n * n * T / (ms_gs / 1e3) / 1e9
    return {"workload": "diff7 as source vs builtin (512^3 FP32 x50); Gray-Scott source 4096^2 x2 FP32 x100",
            "diff7_source_ms": ms_src, "diff7_builtin_ms": ms_blt,
            "source_over_builtin_time": ms_src / ms_blt,
            "gray_scott_ms": ms_gs, "gray_scott_point_updates_per_s": n * n * T / (ms_gs / 1e3),
            "gray_scott_sweeps_per_launch": _sweeps_per_launch(L, g2, gs, f, fo, fw, T),
            "gray_scott_effective_GBps": gbps, "gray_scott_effective_frac": gbps / peak}


def form_batch(L, LI, torch, dev, peak):
    shapes, kinds = LI.batch_shapes(1003, 512)
    grids, ins, outs, works = [], [], [], []
    off = 512 * 3
    for (ny, nx), k in zip(shapes, kinds):
        g = L.Grid((ny, nx), "f32", halo=1)
        g.set_boundaries([k, k])
        grids.append(g)
        ins.append(torch.from_numpy(LI.uniform(1003, ny * nx, off).astype(np.float32).reshape(ny, nx)).to(dev))
        off += ny * nx
    outs = [torch.empty_like(x) for x in ins]
    works = [torch.empty_like(x) for x in ins]
    s = L.Stencil.builtin("jacobi5", 0.2)
    T = 20
    pts = sum(a * b for a, b in shapes)
    wsb = torch.empty(L.batch_workspace_size(grids, s), dtype=torch.uint8, device=dev)
    best, _ = L.autotune_batch(grids, s, ins, outs, works, T, workspace=wsb)  # library autotuner
    tx, ty, k = best.tile_x, best.tile_y, best.tsteps
    # cfg None: lope_apply_batch takes the tuned choice from the autotuner cache
    ms = _time(torch, lambda: L.apply_batch(grids, s, ins, outs, works, T, None, wsb), reps=5)
    per1 = L.Launch(2, 64, 32, 1, -1)

    def per_grid():
        for g, i, o, w in zip(grids, ins, outs, works):
            L.apply(g, s, i, out=o, work=w, nsteps=T, launch=per1)

    ms_pg = _time(torch, per_grid, reps=2)
    return {"workload": "512 jacobi5 FP32 grids, sides U{64..2048}, mixed periodic/Dirichlet, x20",
            "points": pts, "batched_ms": ms, "batched_updates_per_s": pts * T / (ms / 1e3),
            "batched_choice": {"tile": [tx, ty], "tsteps": k},
            "per_grid_ms": ms_pg, "per_grid_updates_per_s": pts * T / (ms_pg / 1e3),
            "per_grid_launches": 512 * T, "speedup": ms_pg / ms,
            "batched_alg_GBps_effective": 8 * pts * T / (ms / 1e3) / 1e9}


def form_adjoint(L, LI, torch, dev, peak):
    n, T, K = 256, 100, 10
    u0 = torch.from_numpy(LI.uniform_field(1004, (n, n, n)).astype(np.float32)).to(dev)
    tg = torch.from_numpy(LI.normal_field(2004, (n, n, n)).astype(np.float32)).to(dev)
    g = L.Grid((n, n, n), "f32", halo=1)
    s = L.Stencil.builtin("diff7", 0.1)
    o, w = torch.empty_like(u0), torch.empty_like(u0)
    ms_fwd = _time(torch, lambda: L.apply(g, s, u0, out=o, work=w, nsteps=T), reps=5)
    wsb = torch.empty(L.workspace_size(g, s, T, K), dtype=torch.uint8, device=dev)
    gu = torch.empty_like(u0)
    ms_adj = _time(torch, lambda: L.adjoint(g, s, u0, tg, T, K, grad_u0=gu, workspace=wsb), reps=3)
    loss, _, gc = L.adjoint(g, s, u0, tg, T, K, grad_u0=gu, workspace=wsb)
    return {"workload": "diff7 FP32 256^3 periodic x100, loss sum((u_T-target)^2), checkpoint 10",
            "plain_forward_ms": ms_fwd, "fwd_adjoint_ms": ms_adj, "ratio": ms_adj / ms_fwd,
            "loss": loss, "dL_dc": gc}


if __name__ == "__main__":
    main()
