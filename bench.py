"""Throughput benchmark of the FED-FEM hot path on GB300.

Workload (one "step" = one explicit FED-FEM time step, Fig. 1 (iii), over the whole mesh):
the large nonlinear cube, 128^3 trilinear hexahedra (2,097,152 elements, 2,146,689 nodes),
orthotropic k = diag(1, 5, 20)(1 + 0.002 T), c = 500 (1 + 0.001 T), rho = 2700, convection and
radiation on all six faces, 1e5 W/m^3 in the central 1/8, FP32 with a Kahan-compensated
temperature accumulator.  Metric: element-steps/s (whole job, summed over ranks).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (oracle/) as it stands on the host cores, on a
bounded sample of the same workload (at most 100 steps of the 128^3 cube), and prints the same
JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "element-steps/s (128^3 hex nonlinear, FP32+Kahan; FP64 and adjoint/forward alongside)"
UNIT = "element-steps/s"
# algorithmic bytes per element-step (general-mesh operator, each array once per step):
# 28 FP32 conductances + 8 int32 node ids per hexahedron, and per node T r/w (8 B), Kahan
# compensation r/w (8 B), FP64 A (8 B), FP32 Q (4 B)
ELEM_BYTES_FP32 = 28 * 4 + 8 * 4
NODE_BYTES_FP32 = 8 + 8 + 8 + 4
ELEM_BYTES_FP64 = 28 * 8 + 8 * 4
NODE_BYTES_FP64 = 16 + 8 + 8
# the same per linear tetrahedron: 6 conductances + 4 int32 node ids
TET_BYTES_FP32 = 6 * 4 + 4 * 4
TET_BYTES_FP64 = 6 * 8 + 4 * 4
L2_BYTES = 129e6
# the benchmark workload (both arms)
WORKLOAD = ("large_hex_128: 128^3 hex nonlinear cube (orthotropic k(T), c(T), conv+rad on all faces, "
            "central source), FP32 + Kahan")
L2_NOTE = "inputs larger than L2 (element stream > 129 MB), no flush"


def round_dt(dt):
    """The time step both arms use: 0.9 dt_crit rounded to 3 significant digits (the GPU's
    Lanczos and the oracle's power iteration agree far below that rounding)."""
    return float(f"{dt:.3g}")


def workload_config(p, dt, n=128):
    """The config dict of the JSON line, the same in both arms."""
    wl = WORKLOAD if n == 128 else WORKLOAD.replace("128", str(n))
    return {"workload": wl, "elements": int(p.n_elems), "nodes": int(p.n_nodes), "dt": dt, "l2": L2_NOTE,
            "parallelism": "single device (replicas with --gpus N)"}


def host_info():
    """Host cores this process may use and the CPU model."""
    from oracle import oracle as O
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return {"nproc": O.host_threads(), "cpu_model": model}


def oracle_dt(p, threads=0):
    """0.9 dt_crit of problem p from the oracle's power iteration (internal loads over the host
    cores), rounded as the GPU arm rounds its own."""
    from oracle import oracle as O
    m = O.OracleModel(p)
    dtc, _, _ = m.dt_crit(tol=1e-7, max_iter=600, threads=threads)
    return m, round_dt(0.9 * dtc)

# The paper's own timings (Section 4.3): C++ on one thread of an Intel i7-6700 @ 3.40 GHz,
# 0.1 m cube with 40,021 tets / 7,872 nodes, dt = 0.005 s, 2000 steps
PAPER_CUBE_MS = {"temperature_independent": 2.376, "temperature_dependent": 4.656}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class NvmlClockSampler:
    """SM clock and clock-event reasons read through NVML (libnvidia-ml, read-only queries) by a
    thread polling every `period_s` while the timed region runs, so that even a region of a
    millisecond or two gets samples."""

    # clock-event reason bits of nvmlDeviceGetCurrentClocksEventReasons
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown"}

    def __init__(self, index, period_s=0.0002):
        import ctypes as C
        self.C = C
        self.period = period_s
        self.rows = []
        self.stop_flag = False
        self.thread = None
        self.nv = C.CDLL("libnvidia-ml.so.1")
        if self.nv.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.h = C.c_void_p()
        bus = None
        try:
            import torch
            pr = torch.cuda.get_device_properties(index)
            bus = "%08x:%02x:%02x.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
        except Exception:
            bus = None
        rc = self.nv.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), C.byref(self.h)) if bus else 1
        if rc != 0 and self.nv.nvmlDeviceGetHandleByIndex_v2(C.c_uint(index), C.byref(self.h)) != 0:
            raise RuntimeError("no NVML handle")
        mx = C.c_uint()
        self.nv.nvmlDeviceGetMaxClockInfo(self.h, 1, C.byref(mx))  # NVML_CLOCK_SM = 1
        self.max_mhz = float(mx.value)
        fn = getattr(self.nv, "nvmlDeviceGetCurrentClocksEventReasons", None)
        self.reasons_fn = fn if fn is not None else self.nv.nvmlDeviceGetCurrentClocksThrottleReasons

    def sample(self):
        C = self.C
        clk, rs = C.c_uint(), C.c_ulonglong()
        if self.nv.nvmlDeviceGetClockInfo(self.h, 1, C.byref(clk)) == 0 and self.reasons_fn(self.h, C.byref(rs)) == 0:
            self.rows.append((float(clk.value), int(rs.value)))

    def _loop(self):
        while not self.stop_flag:
            self.sample()
            time.sleep(self.period)

    def start(self):
        self.sample()
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.thread.start()

    def stop(self):
        self.stop_flag = True
        if self.thread is not None:
            self.thread.join(timeout=2)
        self.sample()
        try:
            self.nv.nvmlShutdown()
        except Exception:
            pass
        sm = [r[0] for r in self.rows]
        reasons = sorted({nm for _, bits in self.rows for b, nm in self.REASONS.items() if bits & b})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": self.max_mhz, "reasons": reasons,
                "samples": len(sm), "source": "nvml"}


def clock_sampler(index):
    """NVML sampler when libnvidia-ml is available, else nvidia-smi."""
    try:
        return NvmlClockSampler(index)
    except Exception:
        return ClockSampler(index)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm), "source": "nvidia-smi"}


def traffic_from_profile(kernel_src_hash):
    """DRAM bytes per step of the step kernel from the committed ncu summary, or None when the
    kernel's code changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "fed_step_kernel_large_hex.md")
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as fh:
        for line in fh:
            if line.startswith("- ") and ":" in line:
                k, v = line[2:].split(":", 1)
                vals[k.strip()] = v.strip().strip("`")
    if vals.get("step.cu code sha256 (comments and whitespace removed)") != kernel_src_hash:
        return None
    try:
        return float(vals["dram bytes per element-step"])
    except (KeyError, ValueError):
        return None


def src_hash():
    """Hash of the step kernel's code: step.cu with its comments and whitespace removed, so that
    a comment edit does not mark the committed counters stale but any code change does."""
    import hashlib
    import re
    with open(os.path.join(ROOT, "paper_1909_03355_gb300", "csrc", "step.cu")) as fh:
        src = fh.read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    code = " ".join(src.split())
    return hashlib.sha256(code.encode()).hexdigest()[:16]


def algorithmic_bytes(p, precision):
    """Bytes one explicit step must move on problem p (each array once)."""
    hexa = p.conn.shape[1] == 8
    if precision == 32:
        eb = ELEM_BYTES_FP32 if hexa else TET_BYTES_FP32
        nb = NODE_BYTES_FP32
    else:
        eb = ELEM_BYTES_FP64 if hexa else TET_BYTES_FP64
        nb = NODE_BYTES_FP64
    return eb * p.n_elems + nb * p.n_nodes


def time_workload(p, precision, steps, stream, peak, dt=None, warm=20, **plan):
    """Device-resident ms/step of `steps` explicit steps of problem p (CUDA events on the
    launching stream, after `warm` untimed steps), with its algorithmic bandwidth.  With
    energy_audit=True in `plan` the line adds the cumulative energy balance of all the steps."""
    import torch
    from paper_1909_03355_gb300.fedfem import FedFem
    f = FedFem(p, precision=precision, stream=stream, **plan)
    dtc = f.precompute()
    dt = 0.9 * dtc if dt is None else dt
    f.set_dt(dt)
    f.set_T(p.initial_T())
    f.step(warm)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        f.step_async(steps)
        e1.record(stream)
    f.sync()
    ms = e0.elapsed_time(e1) / steps
    info = f.info()
    T = f.get_T()
    balance = None
    if plan.get("energy_audit"):
        S, B, n = f.energy_totals()
        balance = {"steps": n, "stored_change_J": S, "boundary_and_source_in_J": B,
                   "rel_residual": abs(S - B) / abs(B) if B else None}
    f.close()
    nbytes = algorithmic_bytes(p, precision)
    gbs = nbytes / (ms * 1e-3) / 1e9
    out = {"precision": "f32+kahan" if precision == 32 else "f64", "steps": steps, "ms_per_step": ms,
           "value": p.n_elems / (ms * 1e-3), "unit": UNIT, "dt": dt, "dt_crit": dtc,
           "algorithmic_MB_per_step": nbytes / 1e6, "achieved_GBps": gbs, "hbm_frac": gbs / peak,
           "working_set": "L2-resident" if nbytes < L2_BYTES else "larger than L2",
           "grid": info["grid"], "block": info["block"], "chunk": info["chunk"], "scatter": info["scatter"],
           "finite": bool(np.all(np.isfinite(T)))}
    if balance is not None:
        out["energy_balance_since_start"] = balance
    return out


def plan_sweep(p, dt, stream, steps=512):
    """Throughput of the 128^3 step over launch plans: CTA size (consumer threads + the producer
    warp) 128 / 256 / 512, steps per launch 1 / 8 / 64 / 512, colour scatter and the atomic
    variant (device-resident, CUDA events around `steps` steps after a warm-up)."""
    import torch
    from paper_1909_03355_gb300.fedfem import FedFem
    rows = []
    for block in (96, 224, 480):
        for scatter in (0, 1):
            for spl in (1, 8, 64, 512):
                row = {"cta_threads": block + 32, "steps_per_launch": spl,
                       "scatter": "atomic" if scatter else "colour"}
                try:
                    f = FedFem(p, precision=32, stream=stream, block=block, steps_per_launch=spl, scatter=scatter)
                    f.precompute()
                    f.set_dt(dt)
                    f.set_T(p.initial_T())
                    f.step(max(spl, 16))
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    with torch.cuda.stream(stream):
                        e0.record(stream)
                        f.step_async(steps)
                        e1.record(stream)
                    f.sync()
                    us = 1e3 * e0.elapsed_time(e1) / steps
                    info = f.info()
                    f.close()
                    row.update({"us_per_step": us, "value": p.n_elems / (us * 1e-6), "grid": info["grid"],
                                "stages": info["stages"]})
                except Exception as e:  # a plan that does not fit is reported, not timed
                    row["error"] = str(e)[:200]
                rows.append(row)
    return {"workload": "large_hex_128", "steps": steps, "rows": rows}


def dd_workload(stream, n_subs=(2, 4), steps=20):
    """The 128^3 cube as slab sub-domains on one device (one launch per sub-domain and step, then
    the halo exchange): wall time per step and the halo bytes a multi-GPU run would send."""
    import fedfem_inputs as fi
    from paper_1909_03355_gb300.dd import FedFemDD
    p = fi.large_cube(128)
    out = {"workload": "large_hex_128 decomposed", "note": "all sub-domains on one GPU (emulation of the exchange); "
           "multi-GPU scaling is unmeasured on hardware", "rows": []}
    for k in n_subs:
        d = FedFemDD(p, k, precision=32, stream=stream)
        dtc = d.precompute()
        d.set_dt(round_dt(0.9 * dtc))
        d.set_T(p.initial_T())
        d.step(3)
        t0 = time.perf_counter()
        d.step(steps)
        el = time.perf_counter() - t0
        info = d.info()
        d.close()
        out["rows"].append({"n_sub": k, "ms_per_step": 1e3 * el / steps, "value": p.n_elems * steps / el,
                            "halo_bytes_per_step": info["halo_bytes_per_step"], "messages": info["n_messages"],
                            "ghost_elements": info["ghost_elements"], "dt_crit": dtc})
    return out


def extra_workloads(stream, peak, own=None):
    """The paper-shaped cube, the 64^3 nonlinear hex and tet cubes, a long slab and the
    jittered 128^3 cube, each in FP32 + Kahan and (where stated) FP64; the L2-resident ones also
    against the L2 copy bandwidth of own_peaks."""
    import fedfem_inputs as fi
    from oracle import oracle as O
    out = {}
    # paper's 0.1 m cube: 19^3 cells x 6 tets (41,154 tets, 8,000 nodes), dt = 0.005 s, 2000 steps
    pc = fi.paper_cube("tet", 19)
    pdt = 0.005
    g32 = time_workload(pc, 32, 2000, stream, peak, dt=pdt)
    g64 = time_workload(pc, 64, 2000, stream, peak, dt=pdt)
    g32td = time_workload(fi.paper_cube("tet", 19, td=True), 32, 2000, stream, peak, dt=pdt)
    # the same laws given as a two-point table (linear between 37 and 337 deg C, held outside)
    pt = fi.paper_cube("tet", 19)
    pt.table_T, pt.table_fk, pt.table_fc = np.array([37.0, 337.0]), np.array([1.0, 10.0]), np.array([1.0, 4.0])
    g32tab = time_workload(pt, 32, 2000, stream, peak, dt=pdt)
    m = O.OracleModel(pc)
    t0 = time.perf_counter()
    m.run(pc.initial_T(), pdt, 400)
    orc_ms = 1e3 * (time.perf_counter() - t0) / 400
    out["paper_cube"] = {
        "workload": "paper_cube_tet_19: 0.1 m cube, 19^3 cells x 6 tets = 41,154 tets, 8,000 nodes, k = 200 iso, "
                    "rho = 1000, c = 2000, T0 = 37, back face held at 37, 0.2 W per node on front/top/sides, "
                    "dt = 0.005 s, 2000 steps",
        "elements": pc.n_elems, "nodes": pc.n_nodes, "gpu_fp32": g32, "gpu_fp64": g64,
        "gpu_fp32_temperature_dependent": g32td,
        "gpu_fp32_temperature_dependent_table": g32tab,
        "oracle_1core_ms_per_step": orc_ms, "oracle_sample": "400 steps, single-threaded FP64 C oracle",
        "real_time_factor_fp32": pdt / (g32["ms_per_step"] * 1e-3),
        "paper_ms_per_step": PAPER_CUBE_MS,
        "paper_context": "C++, one thread of an Intel i7-6700 @ 3.40 GHz, 40,021 tets / 7,872 nodes (Section 4.3)",
        "note": "k(T), c(T) are evaluated every step by the same kernel; the temperature-dependent run uses the "
                "two-point laws of Section 4.2.2 (k 200 -> 2000, c 2000 -> 8000 between 37 and 337 deg C)"}
    for kind in ("hex", "tet"):
        q = fi.nonlinear_cube(64, kind)
        out[f"nonlinear_{kind}_64"] = {"elements": q.n_elems, "nodes": q.n_nodes,
                                        "gpu_fp32": time_workload(q, 32, 2000, stream, peak),
                                        "gpu_fp64": time_workload(q, 64, 400, stream, peak)}
    sl = fi.slab(2048, 32, 32, Lx=1.0, k=(1.0, 5.0, 20.0), k_lin=0.002, c0=500.0, c_lin=0.001, rho=2700.0,
                 T0=20.0, T_s=100.0)
    out["slab_2048x32x32"] = {"elements": sl.n_elems, "nodes": sl.n_nodes,
                              "gpu_fp32": time_workload(sl, 32, 2000, stream, peak)}
    tc = fi.large_cube(128)
    tc.table_T = np.array([0.0, 100.0, 250.0, 450.0, 650.0])
    tc.table_fk = np.array([1.0, 1.6, 1.2, 2.5, 2.0])
    tc.table_fc = np.array([1.0, 0.8, 1.4, 1.1, 1.6])
    out["large_hex_128_table"] = {"elements": tc.n_elems, "nodes": tc.n_nodes,
                                  "note": "the 128^3 cube with a five-point table for k(T), c(T) instead of the "
                                          "linear laws (nodal factors averaged per element)",
                                  "gpu_fp32": time_workload(tc, 32, 2000, stream, peak)}
    ea = fi.large_cube(128)
    out["large_hex_128_energy_audit"] = {
        "elements": ea.n_elems, "nodes": ea.n_nodes,
        "note": "the 128^3 workload with the energy-audit instantiation of the step kernel (FP64 stored-heat "
                "change and boundary input of every node update, summed per CTA); the balance covers the "
                "warm-up and the timed steps",
        "gpu_fp32": time_workload(ea, 32, 2000, stream, peak, energy_audit=True),
        "gpu_fp64": time_workload(ea, 64, 400, stream, peak, energy_audit=True)}
    jc = fi.large_cube(128, jitter=0.2)
    out["large_hex_128_jitter"] = {"elements": jc.n_elems, "nodes": jc.n_nodes,
                                   "note": "interior nodes jittered by +-0.2 h (seeded): every element differs",
                                   "gpu_fp32": time_workload(jc, 32, 2000, stream, peak)}
    l2 = (own or {}).get("l2_copy_GBps")
    if l2:
        for key, rec in out.items():
            for leg in ("gpu_fp32", "gpu_fp64", "gpu_fp32_temperature_dependent", "gpu_fp32_temperature_dependent_table"):
                r = rec.get(leg) if isinstance(rec, dict) else None
                if isinstance(r, dict) and r.get("working_set") == "L2-resident":
                    r["l2_frac"] = r["achieved_GBps"] / l2
                    r["l2_peak_GBps"] = l2
    out["domain_decomposition_128"] = dd_workload(stream)
    return out


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, world, device="cuda"):
    """Largest x over all ranks: a timed region ends when its slowest rank ends."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_barrier(world, sync=None):
    """Barrier over all ranks followed by a device synchronisation (sync, if given)."""
    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        if sync is not None:
            sync()
    return barrier


def whole_job_rate(units_per_rank, world, seconds):
    """Whole-job throughput: every rank processes units_per_rank units (replicas / weak
    scaling) and the job takes the slowest rank's time."""
    return world * units_per_rank / seconds


def run_reference(args, world, rank):
    """FP64 CPU oracle timed on the host cores (the reference arm): the same workload, time step,
    warm-up and step count as the GPU arm, the oracle's time stepping over all host cores."""
    if rank != 0:
        return
    import fedfem_inputs as fi
    n = 128
    p = fi.large_cube(n)
    m, dt = oracle_dt(p)
    hi = host_info()
    T = p.initial_T()
    steps = max(1, min(args.steps, 2000))
    warm = max(0, min(args.warmup, 200))
    T = m.run(T, dt, warm, threads=0)
    t0 = time.perf_counter()
    T = m.run(T, dt, steps, threads=0)
    el = time.perf_counter() - t0
    v = p.n_elems * steps / el
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": steps, "warmup": warm,
            "ms_per_step": 1e3 * el / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": workload_config(p, dt, n),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": hi["nproc"], "kind": "oracle",
                             "cpu_model": hi["cpu_model"],
                             "sample": f"{steps} explicit steps of the {n}^3 hex problem after {warm} warm-up steps, "
                                       f"FP64 C oracle over {hi['nproc']} host threads (element pass, node gather)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline_sample(dt):
    """Oracle element-steps/s on bounded samples of the 128^3 problem: over all host cores (300
    steps, the reported value) and single-threaded as in the paper (40 steps)."""
    import fedfem_inputs as fi
    from oracle import oracle as O
    p = fi.large_cube(128)
    m = O.OracleModel(p)
    hi = host_info()
    T = p.initial_T()
    out = {}
    for threads, steps in ((0, 300), (1, 40)):
        t0 = time.perf_counter()
        m.run(T, dt, steps, threads=threads)
        el = time.perf_counter() - t0
        out[threads] = (p.n_elems * steps / el, steps)
    v, steps = out[0]
    v1, steps1 = out[1]
    return {"value": v, "unit": UNIT, "cores": hi["nproc"], "kind": "oracle", "cpu_model": hi["cpu_model"],
            "sample": f"{steps} explicit steps of the 128^3 hex problem (dt = {dt} s), FP64 C oracle over "
                      f"{hi['nproc']} host threads",
            "single_thread": {"value": v1, "unit": UNIT, "cores": 1,
                              "sample": f"{steps1} steps of the same problem, single-threaded (the paper's mode)"}}


def own_peaks(stream):
    """Roofline denominators measured with the library's own kernels: copy bandwidth of a working
    set held in L2 (two 24 MB buffers), of one streaming from HBM (two 2 GB buffers), and the FP64
    fused-multiply-add rate."""
    import ctypes as C
    import torch
    from paper_1909_03355_gb300 import capi
    L = capi.load()
    h = int(stream.cuda_stream)
    out = {}
    for name, nbytes, reps in (("l2", 24 << 20, 200), ("hbm", 2 << 30, 5)):
        a = torch.empty(nbytes // 4, dtype=torch.float32, device="cuda")
        b = torch.empty_like(a)
        a.fill_(1.0)
        best = 0.0
        for bps in (2, 4):
            ms = C.c_double()
            if L.fedfem_probe_copy(b.data_ptr(), a.data_ptr(), nbytes, reps, bps, h, C.byref(ms)) == 0:
                best = max(best, 2.0 * nbytes * reps / (ms.value * 1e-3) / 1e9)
        out[f"{name}_copy_GBps"] = best
        del a, b
    ms, fl = C.c_double(), C.c_double()
    if L.fedfem_probe_fp64(20000, 8, h, C.byref(ms), C.byref(fl)) == 0:
        out["fp64_TFLOPs"] = fl.value / (ms.value * 1e-3) / 1e12
    torch.cuda.synchronize()
    out["how"] = ("own vector copy kernel (read + write bytes / time, L2: 2 x 24 MB buffers x 200 passes; HBM: 2 x 2 GB "
                  "x 5 passes); own FP64 kernel, 8 independent FMA chains per thread (2 flops per FMA)")
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=400)
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    world, rank, local = dist_setup(args)

    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch
    import torch.distributed as dist

    import fedfem_inputs as fi
    from paper_1909_03355_gb300.fedfem import FedFem

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")

    barrier = make_barrier(world, torch.cuda.synchronize)

    p = fi.large_cube(args.n)
    stream = torch.cuda.Stream()
    f = FedFem(p, precision=32, stream=stream)
    dtc = f.precompute()
    dt = round_dt(0.9 * dtc)
    f.set_dt(dt)

    # CPU baseline (rank 0, N = 1 only), before the timed GPU work
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample(dt)
    T0 = p.initial_T()
    info = f.info()
    spl = info["steps_per_launch"]

    # ---- device-resident throughput (inputs in HBM), per-launch CUDA events on the stream
    f.set_T(T0)
    f.step(args.warmup)
    K = args.steps
    n_launch = int(math.ceil(K / spl))
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(n_launch + 1)]
    clocks = clock_sampler(local)
    clocks.start()
    barrier()
    t_wall = time.perf_counter()
    with torch.cuda.stream(stream):
        ev[0].record(stream)
        done = 0
        for i in range(n_launch):
            k = min(spl, K - done)
            f.step_async(k)
            done += k
            ev[i + 1].record(stream)
    stream.synchronize()
    f.sync()
    barrier()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    durs = [ev[i].elapsed_time(ev[i + 1]) for i in range(n_launch)]
    ms = sum(durs)
    ms = max_over_ranks(ms, world)
    E, N = p.n_elems, p.n_nodes
    value = whole_job_rate(E * K, world, ms * 1e-3)

    # roofline of the step kernel: algorithmic bytes per launch / average launch duration
    bytes_step = ELEM_BYTES_FP32 * E + NODE_BYTES_FP32 * N
    # per-launch step counts (the last launch may be partial); the roofline uses the full
    # launches when there are any, else all launches, with their own step counts
    steps_of = [min(spl, K - i * spl) for i in range(n_launch)]
    sel = [i for i in range(n_launch) if steps_of[i] == spl] or list(range(n_launch))
    launch_steps = sum(steps_of[i] for i in sel) / len(sel)
    avg_launch_ms = sum(durs[i] for i in sel) / len(sel)
    achieved = bytes_step * launch_steps / (avg_launch_ms * 1e-3) / 1e9
    peak, peak_kind = peaks()
    tr = traffic_from_profile(src_hash())

    # ---- end to end through the C ABI with host buffers (H2D of T0, D2H of T inside), both in
    # pinned host memory
    T0_pin = torch.from_numpy(np.ascontiguousarray(T0, dtype=np.float64)).pin_memory()
    Tout_pin = torch.empty(N, dtype=torch.float64, pin_memory=True)
    barrier()
    torch.cuda.synchronize()
    te = time.perf_counter()
    f.set_T(T0_pin.numpy())
    f.step(K)
    Tout = f.get_T(out=Tout_pin.numpy())
    e2e_s = time.perf_counter() - te
    e2e_s = max_over_ranks(e2e_s, world)
    e2e_v = whole_job_rate(E * K, world, e2e_s)
    assert np.all(np.isfinite(Tout))

    # ---- FP64 form on the same workload
    f64 = FedFem(p, precision=64, stream=stream)
    f64.precompute()
    f64.set_dt(dt)
    f64.set_T(T0)
    f64.step(20)
    K64 = args.fp64_steps
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    with torch.cuda.stream(stream):
        e0.record(stream)
        f64.step_async(K64)
        e1.record(stream)
    f64.sync()
    ms64 = e0.elapsed_time(e1)
    ms64 = max_over_ranks(ms64, world)
    v64 = whole_job_rate(E * K64, world, ms64 * 1e-3)
    bytes64 = ELEM_BYTES_FP64 * E + NODE_BYTES_FP64 * N
    # precision policy: the FP32 + Kahan form against the FP64 form after the same steps (untimed)
    T64 = f64.get_T()
    f64.close()
    f.set_T(T0)
    f.step(20 + K64)
    T32 = f.get_T()
    # energy balance of the FP32 run's last step (stored heat change vs boundary and source
    # input, both summed in FP64 from the FP32 states)
    S_e, B_e = f.energy()
    f.close()
    prec = {"steps": 20 + K64, "rel_linf": float(np.max(np.abs(T32 - T64)) / np.max(np.abs(T64))),
            "rel_linf_of_change": float(np.max(np.abs(T32 - T64)) / max(np.max(np.abs(T64 - T0)), 1e-300)),
            "rel_l2_eq30": float(np.linalg.norm(T32 - T64) / np.linalg.norm(T64)),
            "energy_last_step": {"stored_change_J": S_e, "boundary_and_source_in_J": B_e,
                                 "rel_residual": abs(S_e - B_e) / max(abs(B_e), 1e-300)}}

    # ---- adjoint / forward on the 32^3 inverse problem (2000 FP32 steps, 512 sensors sampled
    #      every 10 steps, checkpoints every 100)
    adj = None
    if not args.no_adjoint:
        setup = fi.inverse_problem()
        pi = setup.problem
        torch.cuda.synchronize()
        free_a = torch.cuda.mem_get_info()[0]  # device memory, library allocations included
        fa = FedFem(pi, precision=32, stream=stream)
        dta = 0.9 * fa.precompute()
        fa.set_dt(dta)
        fa.set_T(pi.initial_T())
        torch.cuda.synchronize()
        free_b = torch.cuda.mem_get_info()[0]
        fa.forward_record(200, setup.sensors, 10, 100)  # warm-up
        fa.adjoint(np.zeros((20, len(setup.sensors))))
        fa.set_T(pi.initial_T())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        trc = fa.forward_record(2000, setup.sensors, 10, 100)
        t_fwd = time.perf_counter() - t0
        t0 = time.perf_counter()
        fa.adjoint(np.ones_like(trc))
        t_adj = time.perf_counter() - t0
        torch.cuda.synchronize()
        free_c = torch.cuda.mem_get_info()[0]
        nn_a, ne_a, npe_a = pi.n_nodes, pi.n_elems, pi.npe
        # FP32 run: dL/dtrace, one segment of states, lambda pair + sum mu (FP64), mu (FP32),
        # element slots (FP32), two gradients (FP64), sensor map, FP32 conductances
        sweep_tmp = (trc.size * 8 + 100 * nn_a * 4 + 3 * nn_a * 8 + nn_a * 4 + 2 * ne_a * npe_a * 4 + 2 * ne_a * 8
                     + nn_a * 4 + ne_a * (npe_a * (npe_a - 1) // 2) * 4)
        adj = {"workload": "inverse_32: 32^3 hex, 2000 FP32 steps, 512 sensors every 10 steps, checkpoints every 100",
               "forward_ms": 1e3 * t_fwd, "adjoint_ms": 1e3 * t_adj, "adjoint_over_forward": t_adj / t_fwd,
               "context_device_MB": (free_a - free_b) / 1e6,
               "adjoint_held_device_MB": (free_b - free_c) / 1e6,
               "adjoint_sweep_temporaries_MB": sweep_tmp / 1e6,
               "adjoint_peak_extra_device_MB": (free_b - free_c + sweep_tmp) / 1e6,
               "memory_note": "cudaMemGetInfo deltas (2 MB granularity) for the context after precompute and for "
                              "what forward_record + adjoint keep (checkpoints, trace); the reverse sweep's own "
                              "buffers (one segment of states, lambda pair, mu, sum mu, element F/G slots, two "
                              "gradients, dL/dtrace, sensor map, FP32 conductances) are freed on return and "
                              "counted by size"}
        fa.close()

    # ---- batched scenarios: 256 independent cubes (n ~ U{8..48}, steps ~ U{500..5000}) in one
    #      captured CUDA graph; plan picked by the autotuner on a reduced batch
    batched = None
    if not args.no_batch:
        from paper_1909_03355_gb300.batch import FedFemBatch
        from paper_1909_03355_gb300.tune import BATCH_CANDIDATES, autotune
        scs = fi.batched_scenarios(256)
        small = fi.batched_scenarios(24, seed=44, steps_lo=50, steps_hi=500)
        best, tuned = autotune(lambda **pl: FedFemBatch(small, stream=stream, **pl), BATCH_CANDIDATES,
                               lambda b: b.run(), reps=1)
        fb = FedFemBatch(scs, stream=stream, **best)
        fb.run()  # warm-up replay
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            fb.run()
            e1.record(stream)
        torch.cuda.synchronize()
        bms = e0.elapsed_time(e1)
        tdone, es, _ = fb.times()
        batched = {"workload": "256 cubes, n ~ U{8..48} bricks per edge, steps ~ U{500..5000}, FP32 + Kahan, seed 4",
                   "elements": int(sum(q.n_elems for q in scs)), "element_steps": es,
                   "value": whole_job_rate(es, world, max_over_ranks(bms, world) * 1e-3), "unit": UNIT,
                   "ms": bms,
                   "completion_ms_p50": float(np.percentile(tdone, 50)) / 1e6,
                   "completion_ms_p99": float(np.percentile(tdone, 99)) / 1e6,
                   "plan": best, "tuned": [[r[0], None if r[1] == float("inf") else r[1]] for r in tuned]}
        fb.close()

    own = own_peaks(stream) if rank == 0 else None
    # FP64 form against the FP64 rate: FP64 instructions per element-step, counted from the
    # kernel: per hexahedron 8 adds (mean T), 28 x (subtract + 2 FMA) for the pair loads, 2 for
    # the law and 8 scalings = 102; per node about 24 (update with the IEEE division sequence)
    fp64_instr = 102.0 + 24.0 * N / E
    fp64_alu = None
    if own and own.get("fp64_TFLOPs"):
        rate = fp64_instr * v64 / world  # per GPU
        peak_instr = own["fp64_TFLOPs"] * 1e12 / 2.0
        fp64_alu = {"bound": "alu", "fp64_instructions_per_element_step": fp64_instr,
                    "achieved_T_instr_per_s": rate / 1e12, "peak_T_fma_per_s": peak_instr / 1e12,
                    "frac": rate / peak_instr, "peak_kind": "own FP64 FMA kernel (own_peaks)"}

    sweep = None
    if rank == 0 and not args.no_sweep:
        sweep = plan_sweep(p, dt, stream)

    extras = None
    if rank == 0 and not args.no_extras:
        extras = extra_workloads(stream, peak, own)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": workload_config(p, dt, args.n),
            "plan": {"steps_per_launch": spl, "grid": info["grid"], "block": info["block"], "tiles": info["n_tiles"],
                     "stages": info["stages"], "element_stream_MB": info["elem_bytes"] / 1e6,
                     "ranks": "replicas" if world > 1 else "1 GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "traffic": None if tr is None else tr * E * launch_steps,
                         "algorithmic_bytes_per_launch": bytes_step * launch_steps,
                         "steps_per_timed_launch": launch_steps, "kernel": "fed_step_kernel<float,8,Kahan>",
                         "avg_launch_ms": avg_launch_ms},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": 8 * N / K, "d2h_bytes_per_step": 8 * N / K,
                    "seconds": e2e_s, "host_buffers": "pinned"},
            "gpu_launches": n_launch,
            "clocks": clk,
            "fp64": {"value": v64, "unit": UNIT, "ms_per_step": ms64 / K64, "steps": K64,
                     "achieved_GBps": bytes64 / (ms64 * 1e-3 / K64) / 1e9, "roofline_alu": fp64_alu},
            "own_peaks": own,
            "plan_sweep": sweep,
            "fp32_over_fp64": value / v64,
            "fp32_vs_fp64": prec,
            "adjoint": adj,
            "batched": batched,
            "extras": extras,
            "wall_s": wall,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
