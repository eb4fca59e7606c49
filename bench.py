"""Benchmark: MLUPS of the fused two-component D3Q19 step (fluid + filaments)
and its fraction of the HBM roofline, on the 256x128x64 stripe droplet with
200 nanowires (FP32 storage); FP16/BF16 shifted storage on the same workload
as variants; the FP64 CPU oracle timed on the host cores as the baseline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "2-comp D3Q19 MLUPS & % HBM roofline; FP16-store+batched vs FP32 plain"

# Algorithmic bytes per lattice update of the whole step: 2 components x 19
# directions read and written once (76 s) plus the colour scalars (16 B, 32 B
# in FP64).
ALG_BYTES = {"fp64": 640, "fp32": 320, "fp16": 168, "bf16": 168}

# DRAM bytes (read + write) per launch of the fused kernel from one ncu capture
# (profiles/k_stream_collide_c2_fp32.md), keyed by the hash of the kernel source
# when they were taken, the workload and the tiling; null once any of them differs.
TRAFFIC = {("d5f6b319206d", "c2_256x128x64_stripe_200wires", 6): 362032640 + 305745152}


def kernel_hash():
    """Hash of the fused kernel's source: the k_stream_collide template and the shared
    storage policies it compiles against."""
    d = os.path.join(ROOT, "paper_2607_06794_b300", "csrc")
    src = open(os.path.join(d, "kernels_fluid.cuh")).read()
    i = src.index("k_stream_collide(const InstDev")
    start = src.rindex("template <class S, int TX, int TY>", 0, i)
    end = src.index("\n}\n", i) + 3
    h = hashlib.sha1()
    h.update(src[start:end].encode())
    h.update(open(os.path.join(d, "lbm_internal.cuh"), "rb").read())
    return h.hexdigest()[:12]


def peaks():
    try:
        m = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class _Nvml:
    """The few NVML calls the clock sampler needs, through the driver's libnvidia-ml."""

    CLOCK_SM = 1

    def __init__(self, bus_id=None):
        L = ctypes.CDLL("libnvidia-ml.so.1")
        if L.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        h = ctypes.c_void_p()
        ok = bus_id is not None and L.nvmlDeviceGetHandleByPciBusId_v2(bus_id.encode(), ctypes.byref(h)) == 0
        if not ok and L.nvmlDeviceGetHandleByIndex_v2(0, ctypes.byref(h)) != 0:
            raise RuntimeError("no NVML device handle")
        self.L, self.h = L, h
        self.get_reasons = getattr(L, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            L.nvmlDeviceGetCurrentClocksThrottleReasons

    def sample(self):
        cur, mx, mask = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        if self.L.nvmlDeviceGetClockInfo(self.h, self.CLOCK_SM, ctypes.byref(cur)) != 0:
            return None
        self.L.nvmlDeviceGetMaxClockInfo(self.h, self.CLOCK_SM, ctypes.byref(mx))
        self.get_reasons(self.h, ctypes.byref(mask))
        return cur.value, mx.value, mask.value


class Clocks:
    """SM clocks and throttle reasons sampled during the timed region: NVML polled every
    5 ms from a thread (nvidia-smi every 20 ms when NVML cannot be opened)."""

    REASONS = {"hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40,
               "sw_power_cap": 0x4}

    def __init__(self, bus_id=None):
        import threading
        self.samples, self.maxes, self.reasons = [], [], set()
        self.stop_evt = threading.Event()
        self.p = None
        try:
            self.nv = _Nvml(bus_id)
            self.t = threading.Thread(target=self._poll, daemon=True)
            self.t.start()
        except Exception:
            self.nv = None
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            cmd = ["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "20"]
            if bus_id:
                cmd += ["-i", bus_id]
            try:
                self.p = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
            except Exception:
                self.p = None
            # start timing only once the sampler is running
            t0 = time.time()
            while self.p is not None and time.time() - t0 < 5.0 and os.path.getsize(self.f.name) == 0:
                time.sleep(0.01)

    def _poll(self):
        while not self.stop_evt.is_set():
            try:
                v = self.nv.sample()
                if v is not None:
                    self.samples.append(v[0])
                    self.maxes.append(v[1])
                    for name, bit in self.REASONS.items():
                        if v[2] & bit:
                            self.reasons.add(name)
            except Exception:
                pass
            self.stop_evt.wait(0.005)

    def stop(self):
        if self.nv is not None:
            self.stop_evt.set()
            self.t.join()
            sm, mx = self.samples, self.maxes
            return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                    "reasons": sorted(self.reasons), "samples": len(sm), "source": "nvml 5 ms"}
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock sampling unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm), "source": "nvidia-smi 20 ms"}


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), \
        int(os.environ.get("LOCAL_RANK", 0))


def time_steps(sim, steps):
    import torch
    s = sim.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    sim.step(steps)
    e1.record(s)
    torch.cuda.synchronize()
    sim.sync()
    return e0.elapsed_time(e1)


def make_sim(wl):
    from paper_2607_06794_b300 import Simulation
    sim = Simulation(wl.cfgs)
    wl.setup(sim)
    return sim


def launches_per_step(wl):
    """Kernels of ours per step: fluid, column heights (when the sink can be on),
    and for beads: flags/cells, fields, neighbour list, first kick, one force
    launch per sub-step."""
    n = 1 + (1 if any(c.J0 > 0 and c.evap_start >= 0 for c in wl.cfgs) else 0)
    if any(w is not None and w[0] > 0 for w in wl.wires):
        n += 4 + wl.cfgs[0].substeps
    return n


def oracle_workload(wl, nz=None):
    """The FP64 oracle's state for the same workload: droplet, substrate, wires
    (seeded straight wires inside the droplet, the same count and length)."""
    import numpy as np

    import oracle
    from tests import inputs
    c = wl.cfgs[0]
    nz = c.nz if nz is None else nz
    p = oracle.Params(c.nx, c.ny, nz, tau_R=c.tau_R, tau_B=c.tau_B, beta=c.beta, sigma=c.sigma,
                      J0=c.J0, K=c.K, evap_start=c.evap_start, top_bc=c.top_bc, eps_coh=c.eps_coh,
                      xi=c.xi, gamma=c.gamma)
    fR, fB = oracle.init_droplet(p, c.shape, c.cx, c.cy, c.cz, c.a, c.b, min(c.c, nz - 4), c.width)
    th = wl.thetas[0] if wl.thetas[0] is not None else np.full((c.ny, c.nx), c.theta_deg)
    cot = oracle.cot_map(th)
    beads = None
    if wl.wires[0] is not None:
        nw, L = wl.wires[0]
        nb = int(round(L / c.d0))
        lo = [c.cx - 0.6 * c.a, c.cy - 0.6 * c.b, 2.0]
        hi = [c.cx + 0.6 * c.a, c.cy + 0.6 * c.b, min(0.6 * c.c, nz - 3.0)]
        cen, dirs = inputs.random_filaments(c.seed, nw, nb, c.d0, lo, hi)
        fil, pos, X = inputs.straight_filaments(cen, dirs, nb, c.d0)
        beads = oracle.Beads(fil, pos, X)
    return p, fR, fB, cot, beads


def cpu_baseline(wl, budget_s=12.0):
    """The FP64 oracle on the host cores on whole steps of the same workload."""
    import oracle
    c = wl.cfgs[0]
    p, fR, fB, cot, beads = oracle_workload(wl)
    acc = oracle.Acc()
    oracle.step(p, fR, fB, cot, acc, beads)  # first step: page-in, not timed
    n, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s or n < 2:
        oracle.step(p, fR, fB, cot, acc, beads)
        n += 1
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": round(c.nx * c.ny * c.nz * n / dt / 1e6, 4), "unit": "MLUPS", "cores": cores,
            "kind": "oracle",
            "sample": f"{n} whole FP64 steps of the {wl.name} lattice ({c.nx}x{c.ny}x{c.nz}, "
                      f"{0 if beads is None else beads.n} beads) after one untimed step"}


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle itself on the host cores, same workload and metric."""
    if rank != 0:
        return
    import oracle
    from paper_2607_06794_b300 import workloads
    wl = workloads.WORKLOADS[args.workload]()
    c = wl.cfgs[0]
    # each step is one whole oracle step of the workload; crop z so K+W steps stay ~3 minutes
    per_step = c.nx * c.ny * c.nz / 4.0e6
    nz = c.nz
    if (args.steps + args.warmup) * per_step > 180.0:
        nz = max(8, int(c.nz * 180.0 / ((args.steps + args.warmup) * per_step)))
    p, fR, fB, cot, beads = oracle_workload(wl, nz)
    acc = oracle.Acc()
    for _ in range(args.warmup):
        oracle.step(p, fR, fB, cot, acc, beads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.step(p, fR, fB, cot, acc, beads)
    dt = time.perf_counter() - t0
    mlups = c.nx * c.ny * nz * args.steps / dt / 1e6
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = (f"whole FP64 oracle steps of {c.nx}x{c.ny}x{nz} (the {wl.name} droplet, "
              f"{0 if beads is None else beads.n} beads)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(mlups, 4), "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "lattice": [c.nx, c.ny, nz]},
        "cpu_baseline": {"value": round(mlups, 4), "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(mlups, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}), flush=True)


def reduce_max(v, pg, device):
    """Maximum of a scalar over all ranks (identity without a process group)."""
    if pg is None:
        return v
    import torch
    t = torch.tensor([v], device=device, dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(nodes_per_rank, steps, ms_max, world):
    """Weak scaling: every rank advances its own lattices; the job's throughput is
    all ranks' node updates over the slowest rank's time."""
    return world * nodes_per_rank * steps / (ms_max * 1e-3) / 1e6


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--prec", default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tiling", type=int, default=None,
                    help="use this candidate tiling of the fused kernel instead of autotuning")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch

    from paper_2607_06794_b300 import workloads
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist

    def barrier_max(v):
        return reduce_max(v, pg, "cuda")

    mk = workloads.WORKLOADS[args.workload]
    wl = mk(args.prec) if args.prec else mk()
    prec = wl.cfgs[0].prec
    sim = make_sim(wl)
    sim.step(args.warmup)
    tuned = None
    if args.tiling is not None:
        sim.set_tiling(args.tiling)
        tuned = (args.tiling, None)
        sim.step(3)
    elif not args.no_autotune:
        # part of warm-up: real steps under each candidate tiling
        tuned = sim.autotune(3)
        sim.step(3)
    sim.sync()
    if pg is not None:
        pg.barrier()
    try:
        pr = torch.cuda.get_device_properties(local)
        bus = f"{pr.pci_domain_id:08x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0"
    except Exception:
        bus = None
    clk = Clocks(bus)
    ms = time_steps(sim, args.steps)
    clocks = clk.stop()
    ms = barrier_max(ms)
    ms_step = ms / args.steps
    value = whole_job_mlups(wl.nodes, args.steps, ms, world)

    # roofline of the fused fluid kernel: CUDA events around every launch
    ms_fluid, ms_prof_step = sim.profile_steps(args.steps)
    ms_fluid = barrier_max(ms_fluid)
    hbm, peak_kind = peaks()
    achieved = ALG_BYTES[prec] * wl.nodes / (ms_fluid * 1e-3) / 1e9
    kh = kernel_hash()
    tr = TRAFFIC.get((kh, wl.name, None if tuned is None else tuned[0]))
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(achieved / hbm, 4), "traffic": tr, "peak_kind": peak_kind,
                "kernel": "k_stream_collide", "ms_per_launch": round(ms_fluid, 5),
                "alg_bytes_per_node": ALG_BYTES[prec], "kernel_src": kh,
                "ms_per_step_direct_launch": round(ms_prof_step, 5)}
    sim.sync()

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        c = wl.cfgs[0]
        pops = torch.empty((2, 19, c.nz, c.ny, c.nx), dtype=torch.float64, pin_memory=True)
        sim.read_into(0, "populations", pops)
        accb = torch.empty(6, dtype=torch.float64, pin_memory=True)
        colb = torch.empty((c.nz, c.ny, c.nx), dtype=torch.float64, pin_memory=True)
        # every step: one step, then its budget record copied to pinned host memory
        # behind it on the stream (the host does not wait); the colour field at the end
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.write_from(0, "populations", pops)
        for _ in range(args.steps):
            sim.step(1)
            sim.read_accum_async(0, accb)
        sim.read_into(0, "colour", colb)
        dt = barrier_max(time.perf_counter() - t0)
        assert int(accb[0]) == int(sim.read(0, "accum")[0])
        # the same with a blocking read of the record after every step
        sim.write_from(0, "populations", pops)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for _ in range(args.steps):
            sim.step(1)
            sim.read_into(0, "accum", accb)
        ds = barrier_max(time.perf_counter() - t1)
        e2e = {"value": round(world * wl.nodes * args.steps / dt / 1e6, 2), "unit": "MLUPS",
               "h2d_bytes_per_step": int(pops.numel() * 8 // args.steps),
               "d2h_bytes_per_step": int(32 + colb.numel() * 8 // args.steps),
               "blocking_read_value": round(world * wl.nodes * args.steps / ds / 1e6, 2)}
    steps_done_lp = launches_per_step(wl)
    sim.close()
    del sim
    torch.cuda.empty_cache()

    variants = {}
    if not args.no_variants and args.workload == "c2" and args.prec is None:
        for vp in ("fp16", "bf16"):
            w2 = workloads.droplet_c2(vp)
            s2 = make_sim(w2)
            s2.step(args.warmup)
            if not args.no_autotune:
                s2.autotune(3)
                s2.step(3)
            s2.sync()
            m2 = barrier_max(time_steps(s2, args.steps))
            f2, _ = s2.profile_steps(args.steps)
            mlups2 = world * w2.nodes * args.steps / (m2 * 1e-3) / 1e6
            ach2 = ALG_BYTES[vp] * w2.nodes / (f2 * 1e-3) / 1e9
            variants[vp] = {"value": round(mlups2, 1), "unit": "MLUPS",
                            "speedup_vs_fp32": round(mlups2 / value, 3),
                            "fluid_kernel_GBps": round(ach2, 1), "frac": round(ach2 / hbm, 4),
                            "ms_per_step": round(m2 / args.steps, 5)}
            s2.close()
            del s2
            torch.cuda.empty_cache()

    if not args.no_variants and args.workload == "c2" and args.prec is None:
        # the batched sweep: 64 uneven lattices with wires, FP16 shifted storage, one launch per step
        w4 = workloads.batched_c4("fp16")
        s4 = make_sim(w4)
        s4.step(args.warmup)
        if not args.no_autotune:
            s4.autotune(2)
            s4.step(2)
        s4.sync()
        k4 = max(20, args.steps // 4)
        m4 = barrier_max(time_steps(s4, k4))
        mlups4 = world * w4.nodes * k4 / (m4 * 1e-3) / 1e6
        variants["fp16_batched_c4"] = {"value": round(mlups4, 1), "unit": "MLUPS",
                                       "speedup_vs_fp32": round(mlups4 / value, 3),
                                       "instances": len(w4.cfgs), "nodes": w4.nodes,
                                       "beads": int(sum(s4.nb)), "ms_per_step": round(m4 / k4, 5)}
        s4.close()
        del s4
        torch.cuda.empty_cache()

    if not args.no_variants and args.workload == "c2" and args.prec is None:
        # deposit analysis of Sec. II.B on the c5 wire load (16,000 beads): Kirchhoff network
        # (FP64 CG, one block) and the axial profiles; synchronous calls, wall-clock timed
        from paper_2607_06794_b300 import Simulation
        cfgd, cen, dirs, Xd = workloads.deposit_c5()
        sd = Simulation([cfgd])
        sd.add_nanowires(0, len(cen), 8 * cfgd.d0, cen, dirs)
        sd.write(0, "bead_x", Xd)
        sd.conductivity(0)
        reps = 3
        t0 = time.perf_counter()
        for _ in range(reps):
            cond = sd.conductivity(0)
        t_cond = (time.perf_counter() - t0) / reps
        t0 = time.perf_counter()
        for _ in range(reps):
            sd.profiles(0, 0, 100.0, 412.0, 52, 127.5, 19.0)
        t_prof = (time.perf_counter() - t0) / reps
        variants["deposit_analysis_c5"] = {
            "beads": int(sd.nb[0]), "edges": cond["n_edges"], "kappa": round(cond["kappa"], 6),
            "cg_iterations": cond["iterations"], "conductivity_ms": round(t_cond * 1e3, 3),
            "profiles_ms": round(t_prof * 1e3, 3), "timing": "wall clock of the synchronous call"}
        sd.close()
        del sd
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl)

    if rank == 0:
        c = wl.cfgs[0]
        out = {
            "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32", "fp16": "f16-storage/f32", "bf16": "bf16-storage/f32"}[prec],
            "data": "synthetic",
            "config": {"workload": wl.name, "lattice": [c.nx, c.ny, c.nz], "precision": prec,
                       "nanowires": wl.wires[0][0] if wl.wires[0] else 0,
                       "l2": "inputs larger than L2 (population buffers "
                             f"{2 * 19 * wl.nodes * {'fp64': 8, 'fp32': 4}.get(prec, 2) / 1e6:.0f} MB x2)",
                       "parallelism": f"replicas x{world}",
                       "tiling": None if tuned is None else tuned[0]},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": args.steps * steps_done_lp, "clocks": clocks, "variants": variants,
        }
        print(json.dumps(out), flush=True)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
