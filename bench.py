#!/usr/bin/env python
"""VMC walker-steps/s of the JVB hot path on GB300 (one JSON line on rank 0).

Workload: ethylene-shaped JVB system (16 electrons 8 up / 8 down, 6 nuclei Z = 6,6,1,1,1,1,
6 s + 3 p + 1 d Gaussians per center (M = 126), 6 VB structures / 24 determinants / 8 unique
determinants per spin, e-n + e-e + e-e-n Jastrow, P = 216 parameters), 16384 walkers per GPU,
synthetic seeded inputs.  One step = one VMC sweep of single-electron Metropolis moves over
every walker followed by the evaluation of E_L, dln|Psi|/dp and dE_L/dp for every walker.
The headline form is the mixed one (float bulk, double Slater/ratios/energies); the FP64 form
is reported next to it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "walker-steps/s (E_L + dlnPsi/dp + dE_L/dp), VMC sweep + evaluation"
UNIT = "walker-steps/s"
W_PER_GPU = 16384
REFRESH = 10  # walker-steps between refactorisations of the Slater matrices
SEED = 20220728 + 1

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per walker of the walker kernels
# from one ncu capture (8192 walkers of the same workload; traffic scales with walkers), each
# valid only while that kernel's sources hash to the recorded value (else the bench reports null).
_COMMON_SOURCES = ["walker_common.cuh", "wf_device.cuh", "dsfloat.cuh", "kernels.h", "vbqmc_internal.h"]
WALKER_KERNEL_SOURCES = {"sweep": ["kernels.cu", "sweep_body.cuh"] + _COMMON_SOURCES,
                         "det": ["eval_det.cu", "det_body.cuh"] + _COMMON_SOURCES,
                         "orbitals": ["eval_orbitals.cu", "orbital_body.cuh"] + _COMMON_SOURCES,
                         "jastrow": ["eval_jastrow.cu", "jastrow_body.cuh"] + _COMMON_SOURCES}
PROFILED_TRAFFIC = {
    "sweep": ("282f97f15ec056b95ca54391cd230c827fe9b4dc3b04783db99c8ca6c38daa7d", 10862.5),
    "det": ("2b71d97144b4651efed3caca6ec526642a0828cb1e515851c6e4a118689f42e1", 26410.8),
    "orbitals": ("d68d06277ae1b8dbf8f9209074e417fc21ce06de2e3cdacab233c41ca3dd13dd", 9004.3),
    "jastrow": ("9bb53d641580f851d7480ef8d5c101d8363dfc188579676e4813c39251a35a10", 392.2),
}


def walker_kernel_traffic(kernel, W):
    import hashlib
    if kernel not in PROFILED_TRAFFIC:
        return None
    h = hashlib.sha256()
    for f in WALKER_KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2207_14715_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    sha, per_walker = PROFILED_TRAFFIC[kernel]
    return per_walker * W if h.hexdigest() == sha else None


def workload_config(W, flush=True):
    return {"workload": "ethylene-shaped JVB VMC: 16 e (8/8), 6 nuclei, M=126 Gaussians, 6 structures / "
                        "24 determinants, e-n+e-e+e-e-n Jastrow, P=216, %d walkers per GPU" % W,
            "walkers_per_gpu": W, "electrons": 16, "determinants": 24, "params": 216,
            "l2": "flushed between timed steps (256 MiB write)" if flush else "not flushed",
            "refresh": "Slater matrices refactorised every %d walker-steps; in between the evaluation takes the "
                       "inverses the sweep carries (Sherman-Morrison in double)" % REFRESH}


# --------------------------------------------------------------------------------------
# Algorithmic work per walker-step (documented in the design notes): counted per kernel,
# split into the FP64 and FP32 pipes for each precision form.
# --------------------------------------------------------------------------------------
def work_model(spec, info):
    import numpy as np
    from paper_2207_14715_gb300.systems import NCOMP
    N, Nn = spec.N, spec.Nn
    ncomp = [NCOMP[int(l)] for l in spec.sh_l]
    S = len(ncomp)
    nnz = [(np.nonzero(spec.orb_coef[k])[0].max() - np.nonzero(spec.orb_coef[k])[0].min() + 1)
           if np.any(spec.orb_coef[k]) else 0 for k in range(spec.Norb)]
    det_orbs = sorted(set(int(x) for x in spec.inact) | set(int(x) for x in spec.pairs.ravel()) |
                      set(int(x) for x in spec.unp))
    ev_orbs = sorted(set(det_orbs) | set(int(k) for k in spec.kappa_kl[:, 0]))
    nnz_det = sum(nnz[k] for k in det_orbs)
    nnz_ev = sum(nnz[k] for k in ev_orbs)
    n = spec.n_up
    U = info["U_up"] + info["U_dn"]
    basis_val = S * 6 + 2 * sum(ncomp)          # per point: r^2, exp, N P e per component
    basis_full = S * 6 + 14 * sum(ncomp)        # + gradient and Laplacian per component
    npair = N * (N - 1) // 2
    een_terms = 23
    # ---------------- sweep (N moves from the carried inverses, no factorisation) ----------------
    acc = info.get("acceptance", 0.7)
    sw_row = N * (basis_val + 2 * nnz_det / 2)             # proposed orbital row (own spin's orbitals)
    sw_ratio = N * (U / 2) * 2 * n                          # ratios
    sw_sm = N * acc * (U / 2) * 4 * n * n                   # Sherman-Morrison on accepted moves
    sw64 = sw_ratio + sw_sm
    sw32 = N * ((N - 1) * (30 + Nn * een_terms * 2 * 4) + Nn * 30)   # Jastrow change, old and new
    # ---------------- evaluation with derivatives ----------------
    ev_basis = N * basis_full
    ev_contr_val_det = 2 * N * nnz_det
    ev_contr_rest = 2 * N * (4 * nnz_ev + (nnz_ev - nnz_det))
    # LU + inverse on the refactorising steps (one in REFRESH), the trace tr(A^-1 L) on every step
    ev_lu = U * (2 * n ** 3 + 6 * n * n) / REFRESH + U * 2 * n * n
    ev_jas = npair * (2 * 30) + N * Nn * 30 + 2 * npair * Nn * een_terms * 12
    ev_jderiv = npair * Nn * een_terms * 45 + (npair + N * Nn) * 5 * 10
    ev_kappa = U * 2 * 2 * n * n * len(ev_orbs) + info["n_kappa_entries"] * 2 * n
    ev_orb = ev_basis + ev_contr_val_det + ev_contr_rest
    # per kernel and form: algorithmic flops per walker on the pipe each part runs on
    return {
        "sweep": {"fp64": {"f64": sw64 + sw32 + sw_row, "f32": 0.0}, "mixed": {"f64": sw64, "f32": sw32 + sw_row}},
        "jastrow": {"fp64": {"f64": ev_jas, "f32": 0.0}, "mixed": {"f64": 0.0, "f32": ev_jas}},
        "orbitals": {"fp64": {"f64": ev_orb, "f32": 0.0}, "mixed": {"f64": 0.0, "f32": ev_orb}},
        "det": {"fp64": {"f64": ev_lu + ev_kappa, "f32": 0.0}, "mixed": {"f64": ev_lu, "f32": ev_kappa}},
        "jastrow_deriv": {"fp64": {"f64": ev_jderiv, "f32": 0.0}, "mixed": {"f64": 0.0, "f32": ev_jderiv}},
    }


def measure_peaks(vbqmc, device):
    """ALU peaks measured on this GPU (vbqmc_measure_alu_peaks: FP32 and FP64 FMA chains and
    special-function exponentials over the whole device, CUDA events), with the SM clock sampled
    while the probes ran."""
    sampler = ClockSampler(device)
    sampler.start()
    pk = vbqmc.measure_alu_peaks(device)
    clocks = sampler.stop()
    return {"f32": pk["fp32_tflops"] * 1e12, "f64": pk["fp64_tflops"] * 1e12, "exp": pk["exp_tops"] * 1e12,
            "sms": pk["sms"], "sm_mhz": clocks.get("sm_mhz"), "reasons": clocks.get("reasons", [])}


def file_peaks():
    """HBM copy bandwidth (GB/s) and BF16 GEMM rate (TFLOP/s) measured on this machine's GPUs by the
    environment (MEASURED_PEAKS.json beside this script); the recipe's earlier GB300 figures where
    the file is missing."""
    import json
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]), "source": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


def reblocked_error(x):
    """Standard error of the mean of a correlated series by blocking (Flyvbjerg-Petersen): pairs
    of neighbours are averaged level after level; the error is the largest estimate over the
    levels that keep at least 16 blocks."""
    import numpy as np
    y = np.asarray(x, np.float64)
    errs = []
    while len(y) >= 16:
        errs.append(y.std(ddof=1) / np.sqrt(len(y)))
        y = 0.5 * (y[0:len(y) - len(y) % 2:2] + y[1:len(y) - len(y) % 2:2])
    return max(errs) if errs else float("nan")


# --------------------------------------------------------------------------------------
class ClockSampler:
    """SM clock, its maximum and the clock-event reasons sampled every few milliseconds during
    the timed region: read-only NVML queries (the library nvidia-smi reads) from a polling
    thread, with nvidia-smi itself as the fallback where NVML cannot be loaded."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown"}

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.thread = None
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), "vbqmc_clocks_%d.csv" % os.getpid())

    def _nvml_handle(self):
        import ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            return None, None
        h = ctypes.c_void_p()
        rc = -1
        try:
            import torch
            p = torch.cuda.get_device_properties(self.index)
            bus = "%08x:%02x:%02x.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
            rc = lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(h))
        except Exception:
            rc = -1
        if rc != 0 and lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.index), ctypes.byref(h)) != 0:
            return None, None
        return lib, h

    def _poll(self, lib, h, stop):
        import ctypes
        sm, mx, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        get_rs = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons")
        while not stop.is_set():
            if lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(sm)) == 0 and \
                    lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:
                mask = rs.value if get_rs(h, ctypes.byref(rs)) == 0 else 0
                self.samples.append((float(sm.value), float(mx.value), int(mask)))
            time.sleep(0.005)

    def start(self):
        import threading
        try:
            lib, h = self._nvml_handle()
        except Exception:
            lib, h = None, None
        if lib is not None:
            self.stop_flag = threading.Event()
            self.thread = threading.Thread(target=self._poll, args=(lib, h, self.stop_flag), daemon=True)
            self.thread.start()
            return
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if self.thread is not None:
            self.stop_flag.set()
            self.thread.join(timeout=5)
            if self.samples:
                reasons = sorted({nm for _, _, m in self.samples for bit, nm in self.REASONS.items() if m & bit})
                out = {"sm_mhz": statistics.median(x[0] for x in self.samples),
                       "sm_max_mhz": max(x[1] for x in self.samples), "reasons": reasons,
                       "samples": len(self.samples), "source": "NVML, every 5 ms in the timed region"}
            return out
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                   "samples": len(sm), "source": "nvidia-smi, every 200 ms"}
        return out


def dist_setup():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(x, ws):
    """The slowest rank's time (ranks.max_over_ranks over NCCL)."""
    from paper_2207_14715_gb300 import ranks
    return x if ws == 1 else ranks.max_over_ranks(x, device="cuda")


def cpu_baseline(spec, R_host, seconds_hint=15.0):
    """The oracle as it stands: one walker-step (sweep + E_L + derivatives) on a bounded sample."""
    from oracle import oracle as orc
    cores = os.cpu_count() or 1
    Ws = max(2, min(R_host.shape[0], 2 * cores))
    R = R_host[:Ws].copy()
    t0 = time.perf_counter()
    R, _, _, _ = orc.vmc(spec, R, 1, spec.step, seed=SEED, step0=999, eloc=False, nthreads=cores)
    orc.evaluate(spec, R, derivs=True, nthreads=cores)
    dt = time.perf_counter() - t0
    return {"value": Ws / dt, "unit": UNIT, "cores": min(cores, Ws), "kind": "oracle",
            "sample": "%d walkers x 1 step (sweep + E_L + dlnPsi/dp + dE_L/dp), FP64 CPU oracle, %d threads"
                      % (Ws, min(cores, Ws))}


def run_reference(args, ws, rank):
    """Reference arm: the FP64 CPU oracle, timed on this machine's host cores, on the same workload
    as the GPU arm (each step a bounded sample of its walkers, stated in cpu_baseline)."""
    if rank != 0:
        return
    from paper_2207_14715_gb300 import systems as S
    spec = S.ethylene_vb()
    cores = os.cpu_count() or 1
    R = S.initial_walkers(spec, 2 * cores, SEED)
    for _ in range(args.warmup):
        cpu_baseline(spec, R)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(spec, R))
    dt = time.perf_counter() - t0
    value = sum(v["value"] for v in vals) / len(vals)
    cb = dict(vals[0])
    cb["value"] = value
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic", "config": workload_config(args.walkers, flush=False),
                      "cpu_baseline": cb, "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                                                  "d2h_bytes_per_step": 0}}), flush=True)


def run_ours(args, ws, rank, local):
    import numpy as np
    import torch

    from paper_2207_14715_gb300 import systems as S
    from paper_2207_14715_gb300 import vbqmc

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    spec = S.ethylene_vb()
    info, _, _ = vbqmc.inspect_system(spec)
    W = args.walkers
    P = spec.n_params
    ctx = vbqmc.create(local)
    ctx.set_system(0, spec)
    pk = measure_peaks(vbqmc, local)
    R = torch.tensor(S.initial_walkers(spec, W, SEED + 1000 * rank), device=dev)
    lp = torch.zeros(W, dtype=torch.float64, device=dev)
    sg, el = torch.zeros_like(lp), torch.zeros_like(lp)
    # derivative arrays in each form's bulk type
    Ods = {p: torch.zeros((W, P), dtype=vbqmc.deriv_dtype(p), device=dev) for p in (vbqmc.MIXED, vbqmc.FP64)}
    dEs = {p: torch.zeros_like(Ods[p]) for p in Ods}
    nacc = torch.zeros(W, dtype=torch.int32, device=dev)
    # persistent walker state (Slater inverses, ln|det|, signs) carried from one step to the next
    state = torch.zeros((W, ctx.walker_state_size(0)), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    from paper_2207_14715_gb300 import ranks
    woff = ranks.walker_offset(rank, W)
    step_counter = [0]

    def step(prec, ev=None):
        # one sweep + the evaluation with derivatives in one call; the evaluation takes the
        # inverses the sweep carried and refactorises every REFRESH steps
        k = step_counter[0]
        step_counter[0] += 1
        if ev is not None:
            ev[0].record(stream)
        ctx.vmc_steps(0, prec, R, 1, spec.step, SEED, step0=k, walker_offset=woff, refresh=REFRESH, state=state,
                      state_valid=True, nacc=nacc, logpsi=lp, sign=sg, eloc=el, O=Ods[prec], dEL=dEs[prec])
        if ev is not None:
            ev[1].record(stream)

    # equilibration (untimed), then one evaluation to initialise the walker state
    ctx.vmc_steps(0, vbqmc.MIXED, R, 30, spec.step, SEED, step0=10 ** 6, walker_offset=woff, nacc=nacc)
    ctx.eval_walkers(0, vbqmc.MIXED, R, lp, sg, el, state_out=state)
    torch.cuda.synchronize()
    results = {}
    for name, prec in (("mixed", vbqmc.MIXED), ("fp64", vbqmc.FP64)):
        steps = args.steps if name == "mixed" else max(1, min(args.steps, args.fp64_steps))
        for _ in range(args.warmup):
            step(prec)
        torch.cuda.synchronize()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(steps)]
        nacc.zero_()
        barrier(ws)
        torch.cuda.synchronize()
        sampler = ClockSampler(local) if (rank == 0 and name == "mixed") else None
        if sampler:
            sampler.start()
        # events around each evaluation kernel (read back after every step, outside the
        # device-timed intervals)
        ctx.set_kernel_timing(True)
        ktimes = {key: 0.0 for key in ctx.EVAL_KERNELS}
        t_wall = time.perf_counter()
        for k in range(steps):
            flush.zero_()
            step(prec, evs[k])
            for key, v in ctx.kernel_times().items():
                ktimes[key] += v
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
        ctx.set_kernel_timing(False)
        launches = ctx.last_launch_count()
        barrier(ws)
        clocks = sampler.stop() if sampler else None
        step_ms = sum(e[0].elapsed_time(e[1]) for e in evs)
        eval_ms = sum(ktimes.values())
        sweep_ms = step_ms - eval_ms
        tot_ms = allmax(step_ms, ws)
        kernel_ms = {"sweep": sweep_ms / steps}
        kernel_ms.update({key: v / steps for key, v in ktimes.items()})
        results[name] = {"steps": steps, "ms": tot_ms, "sweep_ms": sweep_ms / steps, "eval_ms": eval_ms / steps,
                         "kernel_ms": kernel_ms, "launches_per_step": launches,
                         "clocks": clocks, "wall_s": t_wall,
                         "acc": float(nacc.double().mean().item()) / (spec.N * steps),
                         "E_mean": float(el.mean().item())}
    # end to end through the C ABI with host buffers (mixed form)
    R_host = torch.empty((W, spec.N, 3), dtype=torch.float64, pin_memory=True)
    R_host.copy_(R.cpu())
    el_host = torch.empty(W, dtype=torch.float64, pin_memory=True)
    e2e_steps = args.steps
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        R.copy_(R_host, non_blocking=True)
        step(vbqmc.MIXED)
        R_host.copy_(R, non_blocking=True)
        el_host.copy_(el, non_blocking=True)
        torch.cuda.synchronize()
    t_e2e = allmax(time.perf_counter() - t0, ws)
    barrier(ws)
    forces = force_timing(ctx, vbqmc, spec, info, R, args.force_steps, pk) if args.force_steps > 0 else None
    eta = efficiency(ctx, vbqmc, spec, R, woff, args.eta_steps) if args.eta_steps > 0 else None
    dmc = dmc_timing(ctx, vbqmc, R, el, args.dmc_steps) if args.dmc_steps > 0 else None
    batched = batched_timing(vbqmc, dev, args.steps) if args.batch_steps > 0 else None
    dmc48 = dmc48_timing(vbqmc, dev, args.dmc48_steps, args.dmc48_walkers) if args.dmc48_steps > 0 else None
    lin = lin_method_timing(ctx, vbqmc, dev, args.steps, file_peaks(), args.lin_samples) if not args.no_lin else None
    barrier(ws)
    if rank != 0:
        return
    model = work_model(spec, dict(info, acceptance=results["mixed"]["acc"]))
    m = results["mixed"]
    value = ws * W * m["steps"] / (m["ms"] * 1e-3)
    f64 = results["fp64"]
    value64 = ws * W * f64["steps"] / (f64["ms"] * 1e-3)
    clocks = m["clocks"] or {}
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    # per-kernel fractions of the measured ALU peaks (the walker path is ALU-bound): each kernel
    # against the pipe its algorithmic work mostly runs on in the mixed form
    km = m["kernel_ms"]
    kroof = {}
    for kname, dur_ms in km.items():
        if dur_ms <= 0:
            continue
        w64 = model[kname]["mixed"]["f64"] * W
        w32 = model[kname]["mixed"]["f32"] * W
        f64_, f32_ = w64 / (dur_ms * 1e-3) / pk["f64"], w32 / (dur_ms * 1e-3) / pk["f32"]
        pipe = "fp64" if f64_ >= f32_ else "fp32"
        ach = (w64 if pipe == "fp64" else w32) / (dur_ms * 1e-3)
        kroof[kname] = {"pipe": pipe, "achieved_tflops": ach / 1e12, "frac": max(f64_, f32_),
                        "other_pipe_frac": min(f64_, f32_), "ms": dur_ms}
    dom = max(km, key=km.get)
    r = kroof[dom]
    roof = {"bound": "alu", "pipe": r["pipe"], "achieved": r["achieved_tflops"],
            "peak": (pk["f64"] if r["pipe"] == "fp64" else pk["f32"]) / 1e12, "unit": "TFLOP/s", "frac": r["frac"],
            "traffic": walker_kernel_traffic(dom, W), "kernel": "%s_kernel<float>" % dom,
            "peak_source": "measured on this GPU by vbqmc_measure_alu_peaks (FP64 %.3f, FP32 %.1f TFLOP/s, "
                           "exp %.2f T/s, %d SMs; SM clock %s MHz during the probes, %.0f MHz during the step)"
                           % (pk["f64"] / 1e12, pk["f32"] / 1e12, pk["exp"] / 1e12, pk["sms"], pk["sm_mhz"],
                              sm_mhz),
            "other_pipe_frac": r["other_pipe_frac"]}
    cb = cpu_baseline(spec, R_host.numpy()) if (ws == 1 and not args.no_cpu_baseline) else None
    bi = W * spec.N * 3 * 8
    bo = W * spec.N * 3 * 8 + W * 8
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": m["steps"], "warmup": args.warmup,
        "ms_per_step": m["ms"] / m["steps"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64 (mixed: float bulk, double Slater LU/inverses/ratios/orbital values/energies)",
        "data": "synthetic (seeded ethylene-shaped system, random-init parameters)",
        "config": workload_config(W),
        "fp64_form": {"value": value64, "unit": UNIT, "ms_per_step": f64["ms"] / f64["steps"],
                      "steps": f64["steps"], "sweep_ms": f64["sweep_ms"], "eval_ms": f64["eval_ms"],
                      "kernel_ms": {k: round(v, 4) for k, v in f64["kernel_ms"].items()}},
        "kernel_ms": {k: round(v, 4) for k, v in km.items()},
        "acceptance": m["acc"], "E_L_mean": m["E_mean"],
        "roofline": roof,
        "kernel_roofline": kroof,
        "efficiency": eta,
        "cpu_baseline": cb,
        "e2e": {"value": ws * W * e2e_steps / t_e2e, "unit": UNIT, "h2d_bytes_per_step": bi,
                "d2h_bytes_per_step": bo,
                "note": "per step: walker positions in, positions and E_L out; the derivative rows O and "
                        "dE_L/dp (2 x 16384 x 216 floats) stay in HBM for the device-side linear method"},
        "linear_method": lin,
        "nuclear_derivs": forces,
        "dmc": dmc,
        "batched": batched,
        "dmc48": dmc48,
        "gpu_launches": m["launches_per_step"] * m["steps"],
        "clocks": {"sm_mhz": clocks.get("sm_mhz"), "sm_max_mhz": clocks.get("sm_max_mhz"),
                   "reasons": clocks.get("reasons", [])},
    }
    print(json.dumps(line), flush=True)


def efficiency(ctx, vbqmc, spec, R0, woff, steps):
    """Statistical efficiency eta = 1 / (sigma^2 t) of the VMC energy in each form: 'steps'
    walker-steps (sweep + evaluation with derivatives, carried inverses, refactorisation every
    REFRESH steps) from the same equilibrated walkers, the walker-averaged E_L of every step,
    sigma = its reblocked standard error of the mean, t = the CUDA-event time of the steps.
    The ratio of the two etas compares the forms at equal statistical error."""
    import numpy as np
    import torch
    W = R0.shape[0]
    dev = R0.device
    out = {}
    for name, prec in (("mixed", vbqmc.MIXED), ("fp64", vbqmc.FP64)):
        R = R0.clone()
        lp, sg, el = (torch.zeros(W, dtype=torch.float64, device=dev) for _ in range(3))
        O = torch.zeros((W, spec.n_params), dtype=vbqmc.deriv_dtype(prec), device=dev)
        dE = torch.zeros_like(O)
        st = torch.zeros((W, ctx.walker_state_size(0)), dtype=torch.float64, device=dev)
        ctx.eval_walkers(0, prec, R, lp, sg, el, state_out=st)
        emean = torch.zeros(steps, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for k in range(steps):
            ctx.vmc_steps(0, prec, R, 1, spec.step, SEED + 7, step0=k, walker_offset=woff, refresh=REFRESH,
                          state=st, state_valid=True, logpsi=lp, sign=sg, eloc=el, O=O, dEL=dE)
            emean[k] = el.mean()
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) * 1e-3
        e = emean.cpu().numpy()
        sig = reblocked_error(e)
        out[name] = {"E_mean": float(e.mean()), "sigma": sig, "seconds": t, "eta": 1.0 / (sig * sig * t)}
    out["steps"] = steps
    out["walkers"] = W
    out["eta_ratio_mixed_over_fp64"] = out["mixed"]["eta"] / out["fp64"]["eta"]
    return out


def force_work(spec, info):
    """Algorithmic flops per walker of the nucleus-derivative kernel (documented in the design
    notes): e-e-n partial derivatives to third order and their assembly per ordered triple
    (i, j, a), e-n terms per (i, a), Gaussian derivatives to third order per (electron, basis
    function), the contraction of 12 derivative values per nonzero coefficient of the
    determinant orbitals, Z_u = B L B once and x_u, y_u per (nucleus, direction)."""
    import numpy as np
    N, Nn, n = spec.N, spec.Nn, spec.n_up
    U = info["U_up"] + info["U_dn"]
    det_orbs = sorted(set(int(x) for x in spec.inact) | set(int(x) for x in spec.pairs.ravel()) |
                      set(int(x) for x in spec.unp))
    nnz_det = sum(int(np.count_nonzero(spec.orb_coef[k])) for k in det_orbs)
    triples = N * (N - 1) * Nn if spec.een_on else 0
    jas = triples * (23 * 6 * 2 * 2 + 12 * 5 * 2 + 3 * 40) + N * Nn * 3 * 40
    basis = N * spec.M * (12 * 3 + 12) + N * len(spec.sh_l) * 3 * 3 * 4 * 4
    contr = N * nnz_det * 12 * 2
    det = U * 2 * 2 * n ** 3 + Nn * U * n * n * 3 * 3 * 2
    return jas + basis + contr + det


def force_timing(ctx, vbqmc, spec, info, R, steps, pk):
    """d ln|Psi|/dR_a and dE_L/dR_a of every walker (one evaluation + the nucleus-derivative
    kernel) in both forms: CUDA events around the call and around a plain evaluation at the
    same positions; the difference is the derivative kernel."""
    import torch
    W = R.shape[0]
    dev = R.device
    lp, sg, el = (torch.zeros(W, dtype=torch.float64, device=dev) for _ in range(3))
    dlp = torch.zeros((W, spec.Nn, 3), dtype=torch.float64, device=dev)
    dE = torch.zeros_like(dlp)
    out = {}
    for name, prec in (("mixed", vbqmc.MIXED), ("fp64", vbqmc.FP64)):
        n = max(3, steps)
        ms = {}
        for what in ("forces", "eval"):
            call = ((lambda: ctx.eval_nuclear_derivs(0, prec, R, lp, sg, el, dlp, dE)) if what == "forces" else
                    (lambda: ctx.eval_walkers(0, prec, R, lp, sg, el)))
            for _ in range(3):
                call()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(n):
                call()
            e1.record()
            torch.cuda.synchronize()
            ms[what] = e0.elapsed_time(e1) / n
        kms = max(ms["forces"] - ms["eval"], 1e-6)
        flops = force_work(spec, info) * W
        pkk = pk["f32" if prec == vbqmc.MIXED else "f64"]
        out[name] = {"walkers_per_s": W / (ms["forces"] * 1e-3), "ms_per_call": ms["forces"],
                     "eval_ms": ms["eval"], "kernel_ms": kms,
                     "kernel_roofline": {"bound": "alu", "pipe": "fp32" if prec == vbqmc.MIXED else "fp64",
                                         "achieved": flops / (kms * 1e-3) / 1e12, "peak": pkk / 1e12,
                                         "unit": "TFLOP/s", "frac": flops / (kms * 1e-3) / pkk}}
    return {"walkers": W, "nuclei": spec.Nn, **out}


def dmc_timing(ctx, vbqmc, R, el, steps, tau=0.005):
    """Fixed-node DMC steps of the mixed form from the equilibrated walkers (population target =
    walker count, capacity 2x): walker-steps/s over the timed steps, CUDA events around the call
    (which synchronizes once per step to read the population)."""
    import torch
    W = R.shape[0]
    buf = torch.zeros((2 * W,) + tuple(R.shape[1:]), dtype=torch.float64, device=R.device)
    buf[:W] = R
    e_t = float(el.mean().item())
    Wc, e_t, _ = ctx.dmc_steps(0, vbqmc.MIXED, buf, W, 3, tau, e_t, W, SEED, step0=1 << 20)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    W1, _, hist = ctx.dmc_steps(0, vbqmc.MIXED, buf, Wc, steps, tau, e_t, W, SEED, step0=(1 << 20) + 3)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    moved = Wc + int(hist["pop"][:-1].sum())
    return {"walker_steps_per_s": moved / (ms * 1e-3), "ms_per_step": ms / steps, "steps": steps, "tau": tau,
            "target": W, "population": [int(x) for x in hist["pop"]],
            "acceptance": hist["accepted"] / max(moved, 1),
            "launches_per_step": (ctx.last_launch_count() - 3) / steps}


def dmc48_timing(vbqmc, dev, steps, W=65536, equil_sweeps=100, warm_steps=20, tau=0.005):
    """The 48-electron system (256 determinants through the reference-determinant tables), W
    (default 65536) walkers, mixed form.  CUDA events around one evaluation (E_L, grad ln|Psi|)
    with the per-kernel times and around one VMC sweep (table sweep).  Then the DMC run of the
    workload: the walkers equilibrated by VMC sweeps (refactorised every 10), E_T = their mean
    E_L, warm_steps untimed DMC steps (tau = 0.005, capacity 1.5x the target), then 'steps' timed
    steps; the population and E_T history of the timed steps and whether the population stayed
    within +-20 % of the target.  walker-steps/s counts the walkers each step moved."""
    import numpy as np
    import torch
    from paper_2207_14715_gb300 import systems as S
    spec = S.dmc48()
    cap = W * 3 // 2
    ctx = vbqmc.create(dev.index or 0)
    ctx.set_system(0, spec)
    buf = torch.zeros((cap, spec.N, 3), dtype=torch.float64, device=dev)
    buf[:W] = torch.tensor(S.initial_walkers(spec, W, SEED + 48), device=dev)
    R0 = buf[:W]
    lp, sg, el = (torch.zeros(W, dtype=torch.float64, device=dev) for _ in range(3))
    g = torch.zeros_like(R0)
    nacc = torch.zeros(W, dtype=torch.int32, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    ctx.vmc_steps(0, vbqmc.MIXED, R0, equil_sweeps, spec.step, SEED, step0=1 << 25, refresh=10, nacc=nacc)
    torch.cuda.synchronize()
    t_equil = time.perf_counter() - t0
    acc = float(nacc.double().sum().item()) / (equil_sweeps * W * spec.N)
    # one table sweep, timed
    e0.record()
    ctx.vmc_steps(0, vbqmc.MIXED, R0, 1, spec.step, SEED, step0=(1 << 25) + equil_sweeps, refresh=1)
    e1.record()
    torch.cuda.synchronize()
    sweep_ms = e0.elapsed_time(e1)
    ctx.set_kernel_timing(True)
    kt = {k: 0.0 for k in ctx.EVAL_KERNELS}
    n = 3
    ev_ms = 0.0
    for _ in range(n):
        e0.record()
        ctx.eval_walkers(0, vbqmc.MIXED, R0, lp, sg, el, g)
        e1.record()
        torch.cuda.synchronize()
        ev_ms += e0.elapsed_time(e1)
        for k, v in ctx.kernel_times().items():
            kt[k] += v
    ctx.set_kernel_timing(False)
    e_vmc = float(el.mean().item())
    Wc, e_t, hist0 = ctx.dmc_steps(0, vbqmc.MIXED, buf, W, warm_steps, tau, e_vmc, W, SEED, step0=1 << 24)
    torch.cuda.synchronize()
    e0.record()
    W1, e_t1, hist = ctx.dmc_steps(0, vbqmc.MIXED, buf, Wc, steps, tau, e_t, W, SEED, step0=(1 << 24) + warm_steps)
    e1.record()
    torch.cuda.synchronize()
    dmc_ms = e0.elapsed_time(e1)
    pops = np.asarray(hist["pop"], np.int64)
    moved = Wc + int(pops[:-1].sum())
    est = hist["sum_wE"] / hist["sum_w"]
    ctx.close()
    return {"electrons": spec.N, "determinants": 256, "unique_per_spin": 70, "walkers": W,
            "vmc_equilibration": {"sweeps": equil_sweeps, "seconds": t_equil, "acceptance": acc,
                                  "E_L_mean_after": e_vmc},
            "sweep_ms": sweep_ms, "sweep_walker_sweeps_per_s": W / (sweep_ms * 1e-3),
            "eval_ms": ev_ms / n, "eval_walkers_per_s": W / (ev_ms / n * 1e-3),
            "eval_kernel_ms": {k: round(v / n, 4) for k, v in kt.items()},
            "dmc_walker_steps_per_s": moved / (dmc_ms * 1e-3), "dmc_ms_per_step": dmc_ms / max(len(pops), 1),
            "tau": tau, "target": W, "warm_steps": warm_steps, "timed_steps": int(len(pops)),
            "population_min_max": [int(pops.min()), int(pops.max())] if len(pops) else None,
            "population_within_20pct": bool(len(pops) and np.all(np.abs(pops / W - 1.0) <= 0.2)),
            "population_every_10": [int(x) for x in pops[::10]],
            "e_trial_every_10": [round(float(x), 4) for x in hist["e_trial"][::10]],
            "estimator_last_10_mean": float(np.mean(est[-10:])) if len(est) else None,
            "acceptance": hist["accepted"] / max(moved, 1)}


def batched_timing(vbqmc, dev, steps):
    """The batched workload (64 random molecules of 2-32 electrons, 256-4096 walkers each) as
    one batch in the mixed form: tuned launch shapes, then steps of one sweep + evaluation with
    derivatives of every system, replayed from the captured graph; walker-steps/s over all
    systems (CUDA events around the timed steps)."""
    import torch
    from paper_2207_14715_gb300 import systems as S
    specs, W = S.batched_workload(64)
    ctx = vbqmc.create(dev.index or 0)
    for k, sp in enumerate(specs):
        ctx.set_system(k, sp)
    R = [torch.tensor(S.initial_walkers(sp, w, SEED + k), device=dev) for k, (sp, w) in enumerate(zip(specs, W))]
    z = lambda: [torch.zeros(w, dtype=torch.float64, device=dev) for w in W]
    lp, sg, el = z(), z(), z()
    O = [torch.zeros((w, sp.n_params), dtype=torch.float32, device=dev) for sp, w in zip(specs, W)]
    dE = [torch.zeros_like(o) for o in O]
    st = [torch.zeros((w, ctx.walker_state_size(k)), dtype=torch.float64, device=dev) for k, w in enumerate(W)]
    batch = vbqmc.Batch(ctx, list(range(len(specs))), W, vbqmc.MIXED)
    batch.tune(R, lp, sg, el)
    args = dict(logpsi=lp, sign=sg, eloc=el, O=O, dEL=dE, state=st)
    batch.vmc_steps(R, 10, 0.3, SEED, step0=1 << 22, refresh=0, **args)   # equilibration, then warm-up
    for k in range(3):
        batch.vmc_steps(R, 1, 0.3, SEED, step0=(1 << 22) + 1 + k, refresh=0, state_valid=True, **args)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = max(3, steps)
    e0.record()
    for k in range(n):
        batch.vmc_steps(R, 1, 0.3, SEED, step0=(1 << 23) + k, refresh=0, state_valid=True, **args)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / n
    launches = ctx.last_launch_count()
    info = batch.info()
    on_tab = [ctx.launch_info(k, vbqmc.MIXED)["tables"] for k in range(len(specs))]
    tables = sum(on_tab)
    # the same step system by system through the single-system call (what the batch replaces)
    def per_system(step0):
        for k in range(len(specs)):
            ctx.vmc_steps(k, vbqmc.MIXED, R[k], 1, 0.3, SEED, step0=step0, refresh=0,
                          state=None if on_tab[k] else st[k], state_valid=not on_tab[k], logpsi=lp[k], sign=sg[k],
                          eloc=el[k], O=O[k], dEL=dE[k])
    per_system((1 << 24))
    torch.cuda.synchronize()
    e0.record()
    for k in range(n):
        per_system((1 << 24) + 1 + k)
    e1.record()
    torch.cuda.synchronize()
    ms_sep = e0.elapsed_time(e1) / n
    batch.close()
    ctx.close()
    # per-electron-pair normalisation: walker-steps/s x mean N^2, comparable across system sizes
    n2 = sum(w * sp.N * sp.N for sp, w in zip(specs, W)) / sum(W)
    return {"systems": len(specs), "walkers": int(sum(W)), "electrons": [min(sp.N for sp in specs),
                                                                       max(sp.N for sp in specs)],
            "systems_on_tables": int(tables), "mean_N2_per_walker": n2,
            "walker_steps_per_s": sum(W) / (ms * 1e-3), "ms_per_step": ms, "launches_per_step": launches,
            "per_system_calls_ms_per_step": ms_sep, "speedup_over_per_system_calls": ms_sep / ms,
            "one_launch": info["one_launch"], "tuned_eval_us": info["tuned_eval_us"],
            "launch_shapes": {k: [info[k]["grid"], info[k]["warps"], info[k]["persist"], info[k]["cap"]]
                              for k in vbqmc.Batch.KINDS}}


def lin_method_timing(ctx, vbqmc, dev, steps, pk, M=1 << 20):
    """Linear-method estimators for M (default 2^20) samples x 400 parameters (mixed form,
    float inputs): time per accumulation with CUDA events, inputs resident in HBM (larger than
    L2); then one timed call split into its four phases (column sums, centring, tensor-core
    products, reduction) with the roofline of each: HBM bytes for the streaming phases, tensor
    flops for the products (algorithmic: 2 x 2 M P^2; issued: three half-precision products per
    pair over the padded 128 x 112 tiles)."""
    import torch
    P = 400
    g = torch.Generator(device=dev)
    g.manual_seed(SEED)
    O = torch.randn((M, P), generator=g, device=dev, dtype=torch.float32)
    dE = 0.3 * torch.randn((M, P), generator=g, device=dev, dtype=torch.float32)
    E = -10.0 + torch.randn(M, generator=g, device=dev, dtype=torch.float64)
    for _ in range(3):  # warm-up (workspace, clocks)
        ctx.accumulate_lin_matrices(vbqmc.MIXED, O, dE, E)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = max(3, steps)
    e0.record()
    for _ in range(n):
        ctx.accumulate_lin_matrices(vbqmc.MIXED, O, dE, E)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / n
    ctx.set_kernel_timing(True)
    ctx.accumulate_lin_matrices(vbqmc.MIXED, O, dE, E)
    ph = list(ctx.kernel_times().values())
    ctx.set_kernel_timing(False)
    flops = 2 * 2.0 * M * P * P  # S and H products
    Pa, Pb, Pm = -(-P // 128) * 128, -(-P // 112) * 112, max(P, 128)
    mma = 3 * 2.0 * M * Pa * (2 * Pb)
    in_bytes = 2 * M * P * 4
    xy_bytes = 2 * Pm * M * 2 * 2  # X and Y, high and low halves, the rows the tensor maps cover
    hbm, bf16 = pk["hbm_gbs"], pk["bf16_tflops"]
    return {"samples": M, "params": P, "ms": ms, "algorithmic_tflops": flops / (ms * 1e-3) / 1e12,
            "input_bytes": in_bytes + M * 8,
            "phases_ms": {"column_sums": ph[0], "centring": ph[1], "tensor_products": ph[2], "reduction": ph[3]},
            "roofline": {
                "column_sums": {"bound": "hbm", "achieved_gbs": in_bytes / (ph[0] * 1e-3) / 1e9,
                                "frac": in_bytes / (ph[0] * 1e-3) / 1e9 / hbm},
                "centring": {"bound": "hbm", "achieved_gbs": (in_bytes + xy_bytes) / (ph[1] * 1e-3) / 1e9,
                             "frac": (in_bytes + xy_bytes) / (ph[1] * 1e-3) / 1e9 / hbm},
                "tensor_products": {"bound": "tensor", "issued_tflops": mma / (ph[2] * 1e-3) / 1e12,
                                    "frac_issued": mma / (ph[2] * 1e-3) / 1e12 / bf16,
                                    "algorithmic_tflops": flops / (ph[2] * 1e-3) / 1e12,
                                    "frac_algorithmic": flops / (ph[2] * 1e-3) / 1e12 / bf16,
                                    "peak": bf16, "peak_note": "%s BF16 burst (f16 runs at the BF16 rate)" % pk["source"]},
                "hbm_peak_gbs": hbm}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--walkers", type=int, default=W_PER_GPU)
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-lin", action="store_true")
    ap.add_argument("--lin-samples", type=int, default=1 << 20, help="samples of the linear-method timing")
    ap.add_argument("--dmc-steps", type=int, default=5, help="timed DMC steps (0: skip)")
    ap.add_argument("--batch-steps", type=int, default=3, help="batched-workload timing (0: skip)")
    ap.add_argument("--force-steps", type=int, default=3, help="nucleus-derivative timing (0: skip)")
    ap.add_argument("--eta-steps", type=int, default=200, help="steps of the efficiency comparison (0: skip)")
    ap.add_argument("--dmc48-steps", type=int, default=100, help="timed DMC steps of the 48-electron system (0: skip)")
    ap.add_argument("--only-dmc48", action="store_true", help="run only the 48-electron DMC leg (long runs)")
    ap.add_argument("--only-lin", action="store_true", help="run only the linear-method leg (profiling)")
    ap.add_argument("--only-batch", action="store_true", help="run only the batched-workload leg (profiling)")
    ap.add_argument("--dmc48-walkers", type=int, default=65536, help="walkers of the 48-electron timing")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        ws = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        run_reference(args, ws, rank)
        return
    ws, rank, local = dist_setup()
    if args.only_dmc48:
        import torch
        from paper_2207_14715_gb300 import vbqmc
        torch.cuda.set_device(local)
        sampler = ClockSampler(local)
        sampler.start()
        out = dmc48_timing(vbqmc, torch.device("cuda", local), args.dmc48_steps, args.dmc48_walkers)
        out["clocks"] = sampler.stop()
        print(json.dumps({"dmc48": out}), flush=True)
        return
    if args.only_lin or args.only_batch:
        import torch
        from paper_2207_14715_gb300 import vbqmc
        torch.cuda.set_device(local)
        dev = torch.device("cuda", local)
        if args.only_lin:
            ctx = vbqmc.create(local)
            out = {"linear_method": lin_method_timing(ctx, vbqmc, dev, args.steps, file_peaks(), args.lin_samples)}
            ctx.close()
        else:
            out = {"batched": batched_timing(vbqmc, dev, args.steps)}
        print(json.dumps(out), flush=True)
        return
    run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
