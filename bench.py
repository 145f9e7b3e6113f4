"""Benchmark of the IGR Euler step on one GB300 (or N independent replicas).

Workload: the many-jet plume, 1024 x 1024 x 2048 cells (2.15e9), 33 Mach-3
inflow jets on z = 0, outflow elsewhere, alpha = dx^2, 5 Jacobi sweeps per
stage, CFL 0.4. A step is one full SSP-RK3 step (3 stages x [source, 5
sweeps, flux/divergence/RK] plus the on-device dt), so the metric is grid
cell-updates per second including the Sigma solve. The headline form is the
16-bit form that meets the workload's accuracy target (2e-3 relative L2 per
field against FP64): FP32 arithmetic, the state in FP32, RK stage increments,
Sigma and b in FP16. Plain FP32 and the form that stores the whole state in
FP16 (half the memory; it misses the target on the momentum) are measured
beside it.

Timing: W warm-up steps, then K steps between a barrier and device
synchronisation, CUDA events on the solver's stream, max over ranks. The
state (21-43 GB) is far larger than L2, so nothing is reused across steps.
Per-kernel CUDA events inside the same timed region give each kernel's
average launch time for the roofline line.

--impl reference times the FP64 CPU oracle (the reference arm of this
benchmark) on the host cores, on a bounded crop of the same workload.
"""
import argparse
import hashlib
import re
from dataclasses import replace
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2505_07392_gb300 import inputs  # noqa: E402

METRIC = "grid cell-updates/s per RK step incl. Σ solve; % HBM roofline; plain vs 16-bit"
FALLBACK_HBM_GBS = 6800.0

# DRAM bytes per cell of one launch from an ncu capture of each kernel on the
# plume workload, keyed by a hash of the kernel source they were taken with;
# a changed source makes the figure stale (reported as null).
# Warp instructions per cell of the dominant kernel (ncu smsp__inst_executed.sum
# over the cells of one launch, mean of the three stage launches), for the
# issue roofline; tied to the kernel source like the traffic.
# Both from ncu captures of the flux kernel on the 512 x 512 x 128 plume,
# mean of the three stage launches of one step.
NCU_INSTR = {
    "flux_f16inc": {"warp_instr_per_cell": 21.159, "src": "475b84c12d696731"},
    "flux_f16": {"warp_instr_per_cell": 22.945, "src": "8eb9327fb53b00ea"},
    "flux_f32": {"warp_instr_per_cell": 20.479, "src": "8eb9327fb53b00ea"},
}

NCU_TRAFFIC = {
    "flux_f16inc": {"bytes_per_cell": 44.333, "src": "475b84c12d696731"},
    "flux_f16": {"bytes_per_cell": 29.105, "src": "8eb9327fb53b00ea"},
    "flux_f32": {"bytes_per_cell": 58.879, "src": "8eb9327fb53b00ea"},
}


def kernel_source_hash():
    """First 16 hex digits of the SHA-256 of igr_kernels.cu and igr_internal.h
    with comments removed and whitespace collapsed: a change of the code makes
    the ncu figures above stale, a change of a comment does not."""
    h = hashlib.sha256()
    for f in ("igr_kernels.cu", "igr_internal.h"):
        src = open(os.path.join(ROOT, "paper_2505_07392_gb300", "csrc", f)).read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, pci_bus_id=None):
        self.proc = None
        self.path = None
        self.pci = pci_bus_id

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.pci:
                cmd.insert(1, f"--id={self.pci}")
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9], _num(parts[3])))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        sm = sorted(r[0] for r in rows)
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        power = sorted(r[3] for r in rows if r[3] is not None)
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows),
                "power_w": power[len(power) // 2] if power else None}


def _num(x):
    try:
        return float(x)
    except ValueError:
        return None


# ------------------------------------------------------------------ GPU arm

def plume_case(args):
    if args.size:
        return inputs.plume(*args.size, steps=args.steps)
    return inputs.plume(steps=args.steps)


def make_case(args):
    """(case, workload description) of --workload (the plume by default),
    with the scheme options --order and --sigma-solver."""
    c, desc = _base_case(args)
    opts = {}
    if args.order != 5:
        opts["order"] = args.order
        desc += f", {args.order}rd-order faces"
    if args.sigma_solver == "rbgs":
        opts["sigma_solver"] = 1
        desc += ", red-black Gauss-Seidel sweeps"
    if args.mu or args.zeta:
        opts["mu"], opts["zeta"] = args.mu, args.zeta
        desc += f", viscous (mu={args.mu:g}, zeta={args.zeta:g})"
    return (replace(c, **opts) if opts else c), desc


def _base_case(args):
    if args.workload == "blast":
        n = args.size[0] if args.size else 256
        c = inputs.blast(n)
        return c, f"spherical blast {n}^3, outflow, S={c.sweeps}"
    if args.workload == "density_wave":
        c = inputs.density_wave(args.size[0] if args.size else 32)
        return c, f"periodic density wave {c.nx}^3, S={c.sweeps}"
    c = plume_case(args)
    return c, f"plume {c.nx}x{c.ny}x{c.nz}, 33 Mach-3 jets, S={c.sweeps}"


def fill_initial_state(case, dtype, device):
    import torch
    if not case.jets:
        return torch.from_numpy(inputs.initial_state(case)).to(dtype).to(device)
    q = torch.empty((5, case.nz, case.ny, case.nx), dtype=dtype, device=device)
    zc = max(1, (1 << 27) // (case.nx * case.ny))
    for k0 in range(0, case.nz, zc):
        k1 = min(case.nz, k0 + zc)
        q[:, k0:k1] = inputs.jet_initial_state(case, (k0, k1, 0, case.ny, 0, case.nx), xp=torch,
                                               device=device, dtype=dtype)
    return q


DTYPE_LABEL = {"f16": "f32 compute, f16 storage", "bf16": "f32 compute, bf16 storage",
               "f16inc": "f32 compute, f32 state, f16 stage increments/Sigma/b",
               "bf16inc": "f32 compute, f32 state, bf16 stage increments/Sigma/b",
               "f32": "f32", "f64": "f64"}


def bytes_per_cell(sweeps, precision):
    """Algorithmic bytes moved per cell by each kernel class over one step.

    One storage type of w bytes: the source reads rho, m (4 words) and writes
    b per stage; a Jacobi sweep reads Sigma, rho, b and writes Sigma; the
    flux kernel reads q and Sigma and writes q (11 words in stage 1), and
    also reads the RK base in stages 2 and 3 (16 words each).

    The increment forms (FP32 state, 16-bit increments, Sigma, b and stage
    density): the source reads rho, m of the state (16 B) and, in stages 2
    and 3, their increments (8 B), and writes b and the stage density (4 B);
    a sweep reads Sigma, the stage density and b and writes Sigma (8 B); the
    flux kernel reads the state (20 B) and Sigma (2 B) in every stage, the
    increments (10 B) in stages 2 and 3, and writes increments (10 B) in
    stages 1 and 2 and the FP32 state (20 B) in stage 3; the RK base of its
    own cell is the state already read for the stencil."""
    if precision.endswith("inc"):
        return {"source": 20 + 28 + 28, "jacobi": 3 * sweeps * 8, "flux": 32 + 42 + 52}
    w = 8 if precision == "f64" else 4 if precision == "f32" else 2
    return {"source": 3 * 5 * w, "jacobi": 3 * sweeps * 4 * w, "flux": (11 + 16 + 16) * w}


def igr_state_bytes(case, precision):
    """Bytes of the state q and Sigma of one case."""
    qb = 8 if precision == "f64" else 4 if precision in ("f32", "f16inc", "bf16inc") else 2
    sb = 8 if precision == "f64" else 4 if precision == "f32" else 2
    return case.ncells * (5 * qb + sb)


def run_form(case, precision, steps, warmup, sync_all, e2e_steps=0, host_rk_base=False, forms=None,
             autotune=False):
    """Time `steps` steps of one precision form; returns a result dict."""
    import torch
    from paper_2505_07392_gb300 import igr
    dev = torch.device("cuda", torch.cuda.current_device())
    st_dtype = igr.state_torch_dtype(precision)
    res = {}
    with igr.Solver(case, precision, host_rk_base=host_rk_base) as s:
        q = fill_initial_state(case, st_dtype, dev)
        s.set_state(q)
        del q
        torch.cuda.synchronize()
        if forms:
            s.set_kernel_forms(*forms)
        if autotune:
            s.autotune(reps=2)
        res["tiles"], res["forms"] = s.tiles(), s.kernel_forms()
        s.step(warmup)
        stream = s.stream
        sync_all()
        torch.cuda.synchronize()
        s.profile(True)
        clk = ClockSampler(getattr(torch.cuda.get_device_properties(dev), "pci_bus_id", None))
        clk.start()
        time.sleep(0.3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            s.step(1, sync=False)
        e1.record(stream)
        torch.cuda.synchronize()
        sync_all()
        clocks = clk.stop()
        ms = e0.elapsed_time(e1)
        prof = {name: s.profile_read(k) for name, k in
                (("source", igr.KC_SOURCE), ("jacobi", igr.KC_JACOBI), ("flux", igr.KC_FLUX),
                 ("other", igr.KC_OTHER))}
        s.profile(False)
        s.sync()
        # FP64 diagnostics of the final state (outside the timed region)
        d = s.diagnose()
        res["diag"] = {"sigma_residual": d["sigma_residual"], "rho_min": d["rho_min"],
                       "p_min": d["p_min"], "sigma_absmax": d["sigma_absmax"]}
        res.update(ms=ms, prof=prof, clocks=clocks)
        if e2e_steps:
            res["e2e"] = run_e2e(s, case, precision, e2e_steps, sync_all)
    torch.cuda.empty_cache()
    return res


# NUMA placement of the pinned host buffer of the end-to-end leg: the
# memory policy of the allocating thread (set_mempolicy, by syscall number:
# no libnuma in the image) decides where the pinned pages land.
_SYS_SET_MEMPOLICY = {"x86_64": 238, "aarch64": 237}
_SYS_GET_MEMPOLICY = {"x86_64": 239, "aarch64": 236}
_MPOL_DEFAULT, _MPOL_PREFERRED = 0, 1
_MPOL_F_NODE, _MPOL_F_ADDR = 1, 2


def gpu_numa_node(device):
    """NUMA node of the GPU's PCI device from sysfs, or None (unknown / -1)."""
    import torch
    bus = getattr(torch.cuda.get_device_properties(device), "pci_bus_id", None)
    if not bus:
        return None
    try:
        bus = bus.lower()
        if len(bus.split(":")[0]) > 4:  # 8-digit PCI domain as CUDA prints it
            bus = bus[4:]
        node = int(open(f"/sys/bus/pci/devices/{bus}/numa_node").read())
        return node if node >= 0 else None
    except (OSError, ValueError):
        return None


def _set_mempolicy(mode, node=None):
    import ctypes
    nr = _SYS_SET_MEMPOLICY.get(os.uname().machine)
    if nr is None:
        return False
    libc = ctypes.CDLL(None, use_errno=True)
    if node is None:
        return libc.syscall(nr, mode, None, ctypes.c_ulong(0)) == 0
    mask = (ctypes.c_ulong * 16)()
    mask[node // 64] |= 1 << (node % 64)
    return libc.syscall(nr, mode, mask, ctypes.c_ulong(16 * 64 + 1)) == 0


def page_numa_node(addr):
    """NUMA node holding the page at host address addr, or None."""
    import ctypes
    nr = _SYS_GET_MEMPOLICY.get(os.uname().machine)
    if nr is None:
        return None
    libc = ctypes.CDLL(None, use_errno=True)
    node = ctypes.c_int(-1)
    r = libc.syscall(nr, ctypes.byref(node), None, ctypes.c_ulong(0), ctypes.c_void_p(addr),
                     ctypes.c_ulong(_MPOL_F_NODE | _MPOL_F_ADDR))
    return node.value if r == 0 and node.value >= 0 else None


def run_e2e(s, case, precision, steps, sync_all):
    """The same metric through the C ABI with HOST buffers: every step is one
    igr_step_host call, which copies the conserved state q in from pinned
    host memory, advances one step and copies the new q back out, the
    read-back overlapped with the last stage. Sigma, the warm start of the
    elliptic solve, stays on the device. The pinned buffer is allocated on
    the GPU's NUMA node where sysfs names one (the node its pages landed on
    and the single-copy bandwidths each way are recorded). For the
    breakdown, the same loop as three separate calls (igr_set_conserved,
    igr_step, igr_get_state), each timed on the host clock."""
    import ctypes
    import torch
    from paper_2505_07392_gb300 import igr
    dt = igr.state_torch_dtype(precision)
    node = gpu_numa_node(s.device)
    bound = node is not None and _set_mempolicy(_MPOL_PREFERRED, node)
    try:
        hq = torch.empty((5,) + s.shape, dtype=dt, pin_memory=True)
    finally:
        if bound:
            _set_mempolicy(_MPOL_DEFAULT)
    code = {torch.float16: igr.DT_F16, torch.bfloat16: igr.DT_BF16, torch.float32: igr.DT_F32,
            torch.float64: igr.DT_F64}[dt]
    L = igr.lib()
    pq = ctypes.c_void_p(hq.data_ptr())

    def check(st):
        if st != igr.OK:
            raise igr.IGRError(st, L.igr_last_error(s.h).decode())

    check(L.igr_get_state(s.h, pq, None, code, 0))
    # single-copy bandwidth each way over the whole buffer (the link's rate
    # can differ between a few GiB and the state's size on some boxes)
    flat = hq.view(-1)
    k = flat.numel()
    dbuf = torch.empty(k, dtype=dt, device=s.device)
    bw = {}
    for name, dst, src in (("h2d_gbs", dbuf, flat[:k]), ("d2h_gbs", flat[:k], dbuf)):
        dst.copy_(src, non_blocking=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        dst.copy_(src, non_blocking=True)
        e1.record()
        e1.synchronize()
        bw[name] = round(k * flat.element_size() / (e0.elapsed_time(e1) * 1e-3) / 1e9, 1)
    del dbuf
    for _ in range(2):  # warm-up of the host path
        check(L.igr_step_host(s.h, pq, pq, 1, code))
    sync_all()
    t0 = time.perf_counter()
    for _ in range(steps):
        check(L.igr_step_host(s.h, pq, pq, 1, code))
    sync_all()
    sec = time.perf_counter() - t0
    # breakdown: separate calls (set_conserved and get_state synchronise with
    # host buffers; igr_sync after the step)
    phase = [0.0, 0.0, 0.0]
    nb = 2
    for _ in range(nb):
        ta = time.perf_counter()
        check(L.igr_set_conserved(s.h, pq, code, 0))
        tb = time.perf_counter()
        check(L.igr_step(s.h, 1, 0.0, None))
        check(L.igr_sync(s.h))
        tc = time.perf_counter()
        check(L.igr_get_state(s.h, pq, None, code, 0))
        td = time.perf_counter()
        phase[0] += tb - ta
        phase[1] += tc - tb
        phase[2] += td - tc
    nbytes = hq.numel() * hq.element_size()
    pages = sorted({page_numa_node(hq.data_ptr() + off) for off in (0, nbytes // 2, nbytes - 4096)} - {None})
    return {"sec": sec, "steps": steps, "bytes": nbytes, "pinned": bool(hq.is_pinned()),
            "phase_s": [x / nb for x in phase], "gpu_numa_node": node, "host_numa_nodes": pages,
            "copy": bw}


def roofline_of(case, res, precision, peak, peak_kind):
    bpc = bytes_per_cell(case.sweeps, precision)
    per = {}
    for name in ("flux", "jacobi", "source"):
        n, ms = res["prof"][name]
        if n == 0 or ms <= 0:
            continue
        algo_bytes = bpc[name] * case.ncells * (res["prof_steps"])  # over the timed region
        gbs = algo_bytes / (ms * 1e-3) / 1e9
        per[name] = {"launches": n, "total_ms": ms, "avg_ms": ms / n,
                     "bytes_per_launch": algo_bytes / n, "achieved_gbs": gbs}
    dom = max(per, key=lambda k: per[k]["total_ms"])
    d = per[dom]
    key = f"{dom}_{precision}"
    t = NCU_TRAFFIC.get(key)
    traffic = (t["bytes_per_cell"] * case.ncells if t and t.get("src") == kernel_source_hash() else None)
    return {"bound": "hbm", "kernel": dom, "achieved": round(d["achieved_gbs"], 1), "peak": peak,
            "unit": "GB/s", "frac": round(d["achieved_gbs"] / peak, 4), "traffic": traffic,
            "peak_kind": f"of {peak_kind}"}, per


def issue_roofline(case, res, precision, clocks, sms):
    """The flux kernel against its issue limit: ncu-counted warp instructions
    per cell x cells per launch x launches / CUDA-event time, over the peak of
    `sms` SMs (the device's count) x 4 schedulers x 1 warp instruction per
    clock at the sampled SM clock. None when no count matches the current
    kernel source."""
    t = NCU_INSTR.get(f"flux_{precision}")
    if not t or t.get("src") != kernel_source_hash() or not clocks:
        return None
    n, ms = res["prof"]["flux"]
    if n == 0 or ms <= 0:
        return None
    achieved = t["warp_instr_per_cell"] * case.ncells * n / (ms * 1e-3)
    peak = sms * 4 * clocks["sm_mhz"] * 1e6
    return {"bound": "issue", "kernel": "flux", "achieved": achieved, "peak": peak,
            "unit": "warp-instr/s", "frac": round(achieved / peak, 4),
            "peak_kind": f"{sms} SMs x 4 schedulers x 1 warp instr/clock at the sampled SM clock"}


# ------------------------------------------------------------ batched arm

def run_batch(args, sync_all=lambda: None):
    """64 periodic Taylor-Green instances of uneven size (edges drawn from
    {48,64,80,96,128}) advanced together: each kernel class one grouped
    launch over all instances (largest first), one CUDA graph per step;
    z-chunks and kernel forms autotuned for the batch (igr_autotune_batch)."""
    import torch
    from paper_2505_07392_gb300 import igr
    cases = inputs.tgv_batch(count=args.batch_count)
    st = igr.state_torch_dtype(args.precision)
    tuned = {}
    with igr.Batch(cases, args.precision) as b:
        for c, inst in zip(cases, b.instances):
            inst.set_state(torch.from_numpy(inputs.initial_state(c)).to(st).cuda())
        torch.cuda.synchronize()
        b.autotune(reps=3)
        for c, inst in zip(cases, b.instances):
            tuned.setdefault((c.nx, c.ny, c.nz), (inst.tiles(), inst.kernel_forms()))
        b.step(args.warmup, sync=True)
        sync_all()
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(args.steps)
        e1.record(stream)
        b.sync()
        sync_all()
        ms = e0.elapsed_time(e1)
    cells = sum(c.ncells for c in cases)
    return {"metric": METRIC, "value": cells * args.steps / (ms * 1e-3), "_cells": cells, "unit": "cell-updates/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE_LABEL[args.precision], "data": "synthetic",
            "config": {"workload": f"{len(cases)} periodic Taylor-Green instances, edges "
                                   f"{sorted(set(c.nx for c in cases))}, {cells} cells, S=5",
                       "tiles": {f"{k[0]}^3": v[0] for k, v in tuned.items()},
                       "vec4_forms": {f"{k[0]}^3": v[1] for k, v in tuned.items()},
                       "l2": "state q and Sigma %.2f GB" % (sum(igr_state_bytes(c, args.precision)
                                                                 for c in cases) / 1e9)}}


# ------------------------------------------------------------ CPU baseline

def oracle_sample_case(full, size):
    """Centred crop of the plume at the inflow face: real -z inflow, every jet
    inside, zero-gradient at the cuts."""
    ny, nx, nz = size
    i0, j0 = (full.nx - nx) // 2, (full.ny - ny) // 2
    jets = [(j[0] - i0 * full.dx, j[1] - j0 * full.dx) + tuple(j[2:]) for j in full.jets]
    bc = (inputs.OUTFLOW,) * 4 + (inputs.INFLOW, inputs.OUTFLOW)
    c = inputs.Case("plume_crop", nx, ny, nz, full.dx, alpha=full.alpha, cfl=full.cfl,
                    sweeps=full.sweeps, bc=bc, jets=jets)
    window = (0, nz, j0, j0 + ny, i0, i0 + nx)
    return c, window


def cpu_baseline(full, steps=1, size=(256, 256, 64)):
    import oracle
    if not full.jets:  # the whole (small) grid
        q0 = inputs.initial_state(full)
        oracle.lib()
        t0 = time.perf_counter()
        oracle.run(full, q0, None, nsteps=steps)
        sec = time.perf_counter() - t0
        cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
        return {"value": full.ncells * steps / sec, "unit": "cell-updates/s", "cores": cores,
                "kind": "oracle", "sample": f"the whole {full.nx}x{full.ny}x{full.nz} grid, "
                                            f"{steps} SSP-RK3 step(s) in FP64, {sec:.1f} s"}
    c, window = oracle_sample_case(full, size)
    q0 = inputs.jet_initial_state(full, window)
    oracle.lib()
    t0 = time.perf_counter()
    oracle.run(c, q0, None, nsteps=steps)
    sec = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": c.ncells * steps / sec, "unit": "cell-updates/s", "cores": cores,
            "kind": "oracle",
            "sample": f"{c.nx}x{c.ny}x{c.nz} crop of the plume at the inflow face (all 33 jets), "
                      f"{steps} SSP-RK3 step(s) in FP64, {sec:.1f} s"}


# -------------------------------------------------------------------- main

def max_over_ranks(ms, world, device):
    """The slowest rank's time: every rank contributes its own and all get the
    maximum (a no-op on one rank)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(cells_per_rank, steps, world, ms):
    """Whole-job cell-updates/s: the cells all ranks advanced over the slowest
    rank's time (replicas: every rank advances its own copy of the workload)."""
    return cells_per_rank * steps * world / (ms * 1e-3)


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    forms = ["f16inc", "bf16inc", "f16", "bf16", "f32", "f64"]
    ap.add_argument("--precision", default="f16inc", choices=forms)
    ap.add_argument("--plain", default="f32", help="second form measured beside the headline ('none' = skip)")
    ap.add_argument("--also", nargs="*", default=["f16"], choices=forms,
                    help="further forms measured beside the headline")
    ap.add_argument("--size", type=int, nargs=3, default=None, metavar=("NX", "NY", "NZ"))
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-size", type=int, nargs=3, default=(256, 256, 128))
    ap.add_argument("--cpu-steps", type=int, default=2)
    ap.add_argument("--workload", default="plume", choices=["plume", "tgv_batch", "blast", "density_wave"])
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--order", type=int, default=5, choices=[3, 5], help="face reconstruction order")
    ap.add_argument("--sigma-solver", default="jacobi", choices=["jacobi", "rbgs"])
    ap.add_argument("--mu", type=float, default=0.0, help="shear viscosity (0: Euler)")
    ap.add_argument("--zeta", type=float, default=0.0, help="bulk viscosity")
    ap.add_argument("--forms", type=int, nargs=2, default=None, metavar=("SOURCE", "JACOBI"),
                    help="kernel forms of the source and Jacobi kernels (1: four cells per thread, 0: one)")
    ap.add_argument("--autotune", action="store_true", help="autotune the launch shape before timing")
    ap.add_argument("--host-rk-base", action="store_true",
                    help="keep the RK base q^n in host memory (read over NVLink-C2C)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    world, rank, local = dist_setup(args)
    full, workload = make_case(args)

    if args.impl == "reference":
        if rank != 0:
            return
        # W warm-up steps are accepted for the contract; the oracle keeps no state to warm
        import oracle
        if full.jets:
            c, window = oracle_sample_case(full, tuple(args.cpu_size))
            q = inputs.jet_initial_state(full, window)
            where = f"{c.nx}x{c.ny}x{c.nz} crop of the plume at the inflow face (all 33 jets)"
        else:
            c, q = full, inputs.initial_state(full)
            where = f"the whole {c.nx}x{c.ny}x{c.nz} grid"
        sig = None
        oracle.lib()
        secs = 0.0
        for _ in range(args.steps):
            t0 = time.perf_counter()
            q, sig, _t = oracle.run(c, q, sig, nsteps=1)
            secs += time.perf_counter() - t0
        value = c.ncells * args.steps / secs
        cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
        cb = {"value": value, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
              "sample": f"{where}, {args.steps} SSP-RK3 step(s) in FP64, {secs:.1f} s"}
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "cell-updates/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * secs / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": workload + (" (oracle on a crop)" if full.jets else ""),
                                                "crop": list(args.cpu_size) if full.jets else None},
                "cpu_baseline": cb,
                "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

        def sync_all():
            dist.barrier()
    else:
        def sync_all():
            pass

    from paper_2505_07392_gb300 import build
    build.build()

    if args.workload == "tgv_batch":
        line = run_batch(args, sync_all)
        ms = max_over_ranks(line["ms_per_step"] * args.steps, world, "cuda")
        line.update(value=job_rate(line.pop("_cells"), args.steps, world, ms), ms_per_step=ms / args.steps,
                    n_gpus=world)
        if rank == 0:
            print(json.dumps(line))
        return

    res = run_form(full, args.precision, args.steps, args.warmup, sync_all,
                   e2e_steps=args.e2e_steps, host_rk_base=args.host_rk_base, forms=args.forms,
                   autotune=args.autotune)
    res["prof_steps"] = args.steps
    ms = max_over_ranks(res["ms"], world, "cuda")
    value = job_rate(full.ncells, args.steps, world, ms)
    # end to end: every rank moves its own replica through host memory; the
    # job takes the slowest rank's time and counts every rank's cells and bytes
    e2e_ms = max_over_ranks(res["e2e"]["sec"] * 1e3, world, "cuda") if "e2e" in res else None
    peak, peak_kind = measured_peaks()
    roof, per_kernel = roofline_of(full, res, args.precision, peak, peak_kind)

    others = {}
    for f in args.also:
        if f in (args.precision, args.plain):
            continue
        ro = run_form(full, f, args.steps, args.warmup, sync_all, host_rk_base=args.host_rk_base,
                      forms=args.forms, autotune=args.autotune)
        ro["prof_steps"] = args.steps
        roof_o, _ = roofline_of(full, ro, f, peak, peak_kind)
        ms_o = max_over_ranks(ro["ms"], world, "cuda")
        others[f] = {"value": job_rate(full.ncells, args.steps, world, ms_o), "ms_per_step": ms_o / args.steps,
                     "roofline": roof_o, "clocks": ro["clocks"]}

    plain = None
    if args.plain not in ("", "none") and args.plain != args.precision:
        rp = run_form(full, args.plain, args.steps, args.warmup, sync_all, host_rk_base=args.host_rk_base,
                      forms=args.forms, autotune=args.autotune)
        rp["prof_steps"] = args.steps
        roof_p, _ = roofline_of(full, rp, args.plain, peak, peak_kind)
        ms_p = max_over_ranks(rp["ms"], world, "cuda")
        plain = {"precision": args.plain, "value": job_rate(full.ncells, args.steps, world, ms_p),
                 "ms_per_step": ms_p / args.steps, "roofline": roof_p, "clocks": rp["clocks"]}

    if rank != 0:
        return
    launches = sum(v[0] for v in res["prof"].values())
    state_gb = igr_state_bytes(full, args.precision) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE_LABEL[args.precision],
        "data": "synthetic",
        "config": {"workload": workload, "cells": full.ncells, "precision": args.precision,
                   "sweeps": full.sweeps, "parallelism": f"replicas x{world}",
                   "rk_base": "host memory (NVLink-C2C)" if args.host_rk_base else "device",
                   "z_chunks": list(res["tiles"]), "kernel_forms": list(res["forms"]),
                   "l2": "inputs larger than L2 (state q and Sigma %.1f GB)" % state_gb},
        "gpu_launches": launches,
        "roofline": roof,
        "kernels": {k: {kk: round(vv, 4) if isinstance(vv, float) else vv for kk, vv in v.items()}
                    for k, v in per_kernel.items()},
        "clocks": res["clocks"],
        "diagnostics_fp64": res["diag"],
    }
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    ri = issue_roofline(full, res, args.precision, res["clocks"], sms)
    if ri:
        line["roofline_issue"] = ri
    # energy from the median sampled power, when the timed region is long
    # enough (>= 1 s, >= 5 samples at 200 ms) for the samples to be under load
    clk = res["clocks"]
    if clk and clk.get("power_w") and clk.get("samples", 0) >= 5 and ms >= 1000.0:
        pw = clk["power_w"]
        line["energy"] = {"power_w": pw, "uJ_per_cell_update": pw * (ms / args.steps) * 1e-3 / full.ncells * 1e6}
    if plain:
        line["plain"] = plain
        line["speedup_vs_plain"] = value / plain["value"]
    if others:
        line["other_forms"] = others
    if "e2e" in res:
        e = res["e2e"]
        line["e2e"] = {"value": job_rate(full.ncells, e["steps"], world, e2e_ms), "unit": "cell-updates/s",
                       "h2d_bytes_per_step": e["bytes"] * world, "d2h_bytes_per_step": e["bytes"] * world,
                       "steps": e["steps"], "pinned": e["pinned"], "call": "igr_step_host",
                       "gpu_numa_node": e["gpu_numa_node"], "host_numa_nodes": e["host_numa_nodes"],
                       "copy_gbs": e["copy"],
                       "separate_calls_s_per_step": {"set_conserved": round(e["phase_s"][0], 4),
                                                     "step": round(e["phase_s"][1], 4),
                                                     "get_state": round(e["phase_s"][2], 4)}}
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(full, args.cpu_steps, tuple(args.cpu_size))
    print(json.dumps(line))


if __name__ == "__main__":
    main()
