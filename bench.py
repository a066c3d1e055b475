"""Benchmark of the chi0 / eps^-1 path on GB300.

One step = the whole path over one synthetic system resident in HBM:
wavefunctions -> mixed grid, oscillator strengths rho for every transition,
transition weights, the chi0 contraction for every frequency, and the FP64
Dyson inversion eps~^-1 for every frequency (chi0_compute_rho +
chi0_build_invert, which runs chi0_build_chi0 and chi0_invert_eps as one
pipeline).

Workload (default): the mixed-precision configuration -- cubic cell a = 10
bohr, 8x8x8 k grid, 16 occupied + 184 empty bands, ~2000 plane waves per
state, FFT 48^3, N_G = 1000, q = (1/4, 0, 0), 32 imaginary frequencies on a
Gauss-Legendre grid in [0, 100] eV, complex64 wavefunctions.

Metric: chi0 build throughput in TFLOP/s of the algorithmic Hermitian count
4 N_G (N_G + 1) N_T N_w per step (N_T = 1,507,328 transitions), i.e. the
inverse of the build time; ms_per_step is that build time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = ("precision: a=10 bohr, k 8x8x8, 16+184 bands, ~2000 PW, FFT 48^3, N_G=1000, "
            "q=(1/4,0,0), 32 imaginary GL frequencies in [0,100] eV, complex64 wavefunctions")
METRIC = "chi0(q,w) build throughput (algorithmic Hermitian TFLOP/s) incl. rho and FP64 eps^-1"


def chi0_flops(ng, nt, nw):
    return 4.0 * ng * (ng + 1) * nt * nw


def max_over_ranks(x, dist, device):
    """The largest value of x over all ranks (x itself without a process group):
    the job's time is that of its slowest replica."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_tflops(world, flops_per_step, ms_per_step):
    """Throughput of the whole job: each of the world ranks runs one replica
    of the step (no data-path collective), in the slowest rank's time."""
    return world * flops_per_step / (ms_per_step * 1e-3) / 1e12


# stage -> (binding roof, unit, kernel)
STAGE_ROOF = {"contract": ("tensor", "TFLOP/s", "k_herk_wide"), "rho": ("alu", "TFLOP/s", "k_rho_pairs"),
              "wf_grid": ("alu", "TFLOP/s", "k_wf_to_mixed"), "dyson": ("fp64", "TFLOP/s", "k_gj_update"),
              "weights": ("hbm", "GB/s", "k_prep"), "reduce": ("hbm", "GB/s", "k_tc_reduce")}
# FP32 FMA: 152 SMs x 128 lanes x 2 flop x 1.93 GHz (the clock seen under this load)
FP32_PEAK, FP32_SRC = 75.0, "FP32 FMA: 152 SMs x 128 lanes x 2 flop x 1.93 GHz"
# FP64: the nominal GB300 figure (no measured FP64 peak is available)
FP64_PEAK, FP64_SRC = 1.25, "FP64 nominal (GB300)"
# Stored DRAM traffic per launch (ncu, dram__bytes_read.sum +
# dram__bytes_write.sum) is read from the profile summaries under profiles/:
# lines of the form
#   traffic: <kernel> | <workload> | <bytes per launch> | <source file> <sha256 prefix> | <how>
# A figure is used only while the kernel's source file still has the hash it
# had when the counters were taken; after any change it reads as null.
KERNEL_SOURCE = {"k_herk_bf16x3": "tc.cu", "k_herk_wide": "tc.cu", "k_prep": "tc.cu", "k_rho_pairs": "rho.cu",
                 "k_wf_to_mixed": "rho.cu", "k_gj_update": "dyson.cu", "k_chi0_fp64": "chi0_fp64.cu"}


def source_sha(fname):
    import hashlib
    path = os.path.join(ROOT, "paper_1902_03837_gb300", "csrc", fname)
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def stored_traffic(kernel, workload):
    """(bytes per launch, description) of the stored ncu figure for kernel on
    workload, or (None, reason)."""
    import glob
    src = KERNEL_SOURCE.get(kernel)
    found = None
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(path) as f:
            for line in f:
                if not line.startswith("traffic:"):
                    continue
                parts = [x.strip() for x in line[len("traffic:"):].split("|")]
                if len(parts) < 5 or parts[0] != kernel or parts[1] != workload:
                    continue
                found = (float(parts[2]), parts[3].split(), parts[4], os.path.basename(path))
    if found is None or src is None:
        return None, "no stored ncu figure for this kernel and workload"
    nbytes, (fname, sha), how, where = found
    if fname != src or sha != source_sha(src):
        return None, f"the kernel's source changed since the stored ncu figure ({where})"
    return nbytes, f"{how} ({where}, {fname} {sha})"


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return {"hbm_gbs": p["hbm_gbs"], "bf16_tflops": p["bf16_tflops"],
                "bf16_tflops_sustained": p["bf16_tflops_sustained"], "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "source": "fallback"}


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                self.out, _ = self.p.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5], f[6], f[7], f[8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[2 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


PPA_OMEGA_P = 1.0          # Ha: the plasmon-pole model's second fit point i omega_p (PPAPntXp default)
PPA_ETA_EV = 0.1           # broadening of the model's real-axis evaluation


def ppa_real_freqs(n):
    from synth import HA_EV
    return np.arange(1, n + 1) * (100.0 / n) / HA_EV + 0j


def build_system(kgrid=None, nw=32, real_axis=False, ppa=False, flat=False):
    """The precision workload; kgrid / nw override it for smaller profiling
    runs; real_axis puts its nw frequencies on the real axis instead (evenly
    spaced on (0, 100] eV, broadening 0.1 eV); ppa keeps only the plasmon-pole
    fit points w = 0 and w = i omega_p."""
    import dataclasses
    from synth import HA_EV, cfg_precision, make_system
    spec = cfg_precision(nw=nw)
    if kgrid is not None:
        spec.kgrid = tuple(kgrid)
    if real_axis:
        w = np.arange(1, nw + 1) * (100.0 / nw) / HA_EV
        spec = dataclasses.replace(spec, freqs=tuple(complex(x, 0.0) for x in w), eta=0.1 / HA_EV)
    if ppa:
        spec = dataclasses.replace(spec, freqs=(0j, 1j * PPA_OMEGA_P))
    if flat:
        spec = dataclasses.replace(spec, flat_bands=True)
    return make_system(spec)


def workload_name(args):
    base = _workload_base(args)
    if getattr(args, "real_axis", False):
        base = base.replace(" imaginary GL frequencies in [0,100] eV", " real frequencies on (0,100] eV, eta 0.1 eV")
    if getattr(args, "ppa", None):
        base = base.replace(f"{args.nw} imaginary GL frequencies in [0,100] eV",
                            f"chi0 and eps^-1 at w = 0 and i 1 Ha, Godby-Needs plasmon-pole fit, "
                            f"model on {args.ppa} real frequencies on (0,100] eV, eta 0.1 eV")
    if getattr(args, "bg_terminator", None) is not None:
        base += f", Bruneval-Gonze extrapolar correction at {args.bg_terminator:g} eV"
    if getattr(args, "flat_bands", False):
        base += ", dispersionless bands (every k has the energies of k = 0)"
    if getattr(args, "grouping", 0.0):
        base += f", pole grouping at {args.grouping:g} Ha"
    return base


def workload_tag(args):
    """Short name of the workload for the stored ncu figures."""
    k = "x".join(str(v) for v in (args.kgrid or (8, 8, 8)))
    tag = f"precision k{k} nw{args.nw}"
    if getattr(args, "real_axis", False):
        tag += " real"
    if getattr(args, "ppa", None):
        tag += f" ppa{args.ppa}"
    if getattr(args, "bg_terminator", None) is not None:
        tag += " bg"
    if getattr(args, "precision", "mixed") == "fp64":
        tag += " fp64"
    return tag


def stage_rooflines(args, st_ms, st_bytes, st_flops, pk, nt, ng, nw):
    """Achieved rate of every stage against the roof that binds it, per step:
    rho and the wavefunction transforms against the FP32 (or FP64) pipe and
    HBM, the operand split against HBM, the contraction against the tensor
    cores (algorithmic count), the Dyson step against the FP64 units."""
    out = {}
    fp64 = args.precision == "fp64"
    for st in ("wf_grid", "rho", "weights", "contract", "reduce", "dyson"):
        ms = st_ms[st] / args.steps
        if ms <= 0:
            continue
        sec = ms * 1e-3
        gbs = st_bytes[st] / sec / 1e9
        tfs = st_flops[st] / sec / 1e12
        e = {"ms_per_step": ms, "gbs": gbs, "hbm_frac": gbs / pk["hbm_gbs"], "tflops": tfs}
        if st in ("wf_grid", "rho"):
            peak, src = (FP64_PEAK, FP64_SRC) if fp64 else (FP32_PEAK, FP32_SRC)
            e.update(bound="fp64" if fp64 else "alu", alu_peak=peak, alu_frac=tfs / peak, alu_peak_source=src)
        elif st == "contract":
            if fp64:
                e.update(bound="fp64", alu_peak=FP64_PEAK, alu_frac=tfs / FP64_PEAK, alu_peak_source=FP64_SRC)
            else:
                e.update(bound="tensor", tensor_peak=pk["bf16_tflops_sustained"],
                         tensor_frac=tfs / pk["bf16_tflops_sustained"])
        elif st == "dyson":
            e.update(bound="fp64", alu_peak=FP64_PEAK, alu_frac=tfs / FP64_PEAK, alu_peak_source=FP64_SRC)
        else:
            e.update(bound="hbm")
        out[st] = e
    return out


def _workload_base(args):
    if args.kgrid is None and args.nw == 32:
        return WORKLOAD
    k = "x".join(str(v) for v in (args.kgrid or (8, 8, 8)))
    return WORKLOAD.replace("k 8x8x8", f"k {k}").replace("32 imaginary", f"{args.nw} imaginary")


# ----------------------------------------------------------------------------- CPU baseline (the oracle)

# The CPU baseline leg: the oracle's chi0 on the G_0..G_63 sub-block of the
# benchmark's own system (all transitions, all frequencies), summed over k
# chunks by worker processes, and the oracle's Gauss-Jordan inversion of two
# of the GPU's eps~.  Its time is the reported CPU baseline; its results give
# the error of the GPU path.  The workers are spawned (no GPU state), read the
# system from files the parent writes, and run on every host core but the
# first, which keeps issuing the GPU work.
ERR_G = 64                  # G_0 .. G_63: the real tile (0, 0) of the contraction
_ERR = {}
_SYS_ARRAYS = ("lattice", "kfrac", "npw", "gvec", "coef", "eps", "occ", "q_frac", "freqs")


def _err_init(path, cores):
    """Worker set-up: one thread each, pinned to the worker cores; the
    system's arrays mapped read-only from the files the parent wrote."""
    import pickle
    try:
        os.sched_setaffinity(0, cores)
    except (AttributeError, OSError):
        pass
    with open(os.path.join(path, "system.pkl"), "rb") as f:
        meta = pickle.load(f)
    arrays = {k: np.load(os.path.join(path, k + ".npy"), mmap_mode="r") for k in _SYS_ARRAYS}
    from synth import System
    _ERR["s"] = System(**meta["fields"], **arrays)
    _ERR["G"] = meta["G"]


def _err_chunk(ks):
    import oracle as O
    s = _ERR["s"]
    return O.chi0_tr(s, 0, _ERR["G"], s.freqs, s.eta, ks=ks)


def _err_gj(chi, qg):
    import oracle as O
    return O.eps_inv_gauss_jordan(chi, qg)


class OracleJobs:
    """Worker processes (spawned, one thread each, on every host core but the
    first) that run the oracle for the CPU baseline leg."""

    def __init__(self, system):
        import multiprocessing as mp
        import pickle
        import tempfile
        import oracle as O
        G = O.response_gvectors(system.spec.kgrid, system.q_frac[0], system.ng)
        self.qg = O.qg_norms(system.spec.a, system.q_frac[0], G)
        self.tmp = tempfile.TemporaryDirectory(prefix="chi0_baseline_")
        for k in _SYS_ARRAYS:
            np.save(os.path.join(self.tmp.name, k + ".npy"), np.ascontiguousarray(getattr(system, k)))
        fields = {k: getattr(system, k) for k in ("spec", "omega_cell", "eta", "spin_factor", "fft", "ng")}
        with open(os.path.join(self.tmp.name, "system.pkl"), "wb") as f:
            pickle.dump({"fields": fields, "G": G[:ERR_G]}, f)
        try:
            cores = sorted(os.sched_getaffinity(0))
        except AttributeError:
            cores = list(range(os.cpu_count() or 1))
        work = set(cores[1:]) or set(cores)
        self.nproc = len(work)
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(self.nproc, initializer=_err_init,
                                                     initargs=(self.tmp.name, work))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self.nk = system.nk
        self.chunks = None
        self.gj = []

    def start_chi0(self):
        ks = list(range(self.nk))
        step = max(1, -(-self.nk // (4 * self.nproc)))
        self.t0 = time.perf_counter()
        self.chunks = self.pool.map_async(_err_chunk, [ks[i:i + step] for i in range(0, self.nk, step)])

    def start_gj(self, chi):
        self.gj.append(self.pool.apply_async(_err_gj, (chi, self.qg)))

    def chi0(self):
        parts = self.chunks.get()
        return sum(parts[1:], parts[0]), time.perf_counter() - self.t0

    def gj_results(self):
        return [r.get() for r in self.gj]

    def close(self):
        self.pool.close()
        self.pool.join()
        self.tmp.cleanup()


def rel_fro(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# ----------------------------------------------------------------------------- reference arm

def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample(system, nks, G):
    """The CPU oracle on nks k points (all transitions there, all G, all w)."""
    import oracle as O
    t0 = time.perf_counter()
    O.chi0_tr(system, 0, G, system.freqs, system.eta, ks=list(range(nks)))
    dt = time.perf_counter() - t0
    nt = nks * system.spec.n_occ * (system.nb - system.spec.n_occ)
    return dt, chi0_flops(system.ng, nt, system.freqs.size)


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle as O
    s = build_system(args.kgrid, args.nw)
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], s.ng)
    nks = 4
    vals = []
    for i in range(args.warmup + args.steps):
        dt, fl = oracle_sample(s, nks, G)
        if i >= args.warmup:
            vals.append((dt, fl))
    tot_t = sum(v[0] for v in vals)
    tot_f = sum(v[1] for v in vals)
    value = tot_f / tot_t / 1e12
    cores = cpu_cores()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / len(vals),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": workload_name(args), "sample": f"{nks} of {s.nk} k points per step"},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": f"FP64 numpy oracle, all transitions of {nks} of {s.nk} k points, "
                                   f"all {s.ng} G and {s.freqs.size} frequencies, per step"},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- our arm

def run_ours(args, rank, world, dist):
    import torch
    s = build_system(args.kgrid, args.nw, args.real_axis, ppa=bool(args.ppa), flat=args.flat_bands)
    ng, nw = s.ng, s.freqs.size
    # the plain FP64 form and the CPU baseline on the G_0..G_63 sub-block (with
    # the error against it) are measured on the imaginary-axis workload (rank
    # 0 only); the baseline's workers start here, before any CUDA call
    plain = (rank == 0 and args.precision == "mixed" and not args.ppa and not args.real_axis
             and args.bg_terminator is None and not args.grouping and not args.flat_bands)
    compare = plain and not args.no_compare
    jobs = OracleJobs(s) if (plain and not args.no_cpu_baseline) else None
    import __graft_entry__ as g
    g.build()
    from paper_1902_03837_gb300 import chi0 as lib

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    prec = lib.CHI0_MIXED_BF16X3 if args.precision == "mixed" else lib.CHI0_FP64
    ctx = lib.Chi0.for_system(s, precision=prec, stream=stream.cuda_stream)
    # inputs resident in HBM (device-to-device set keeps the timed region free of host copies)
    gv_d = [torch.from_numpy(np.ascontiguousarray(s.gvec[ik, :s.npw[ik]])).to(dev) for ik in range(s.nk)]
    cf_d = [torch.from_numpy(np.ascontiguousarray(s.coef[ik, :, :s.npw[ik]])).to(dev) for ik in range(s.nk)]
    for ik in range(s.nk):
        ctx.set_wavefunctions(ik, gv_d[ik], cf_d[ik])
    ctx.set_energies(s.eps, s.occ)
    if args.bg_terminator is not None:
        from synth import HA_EV
        ctx.set_bg_terminator(args.bg_terminator / HA_EV)
    if args.grouping:
        ctx.set_pole_grouping(args.grouping)
    inv_d = torch.empty((nw, ng, ng), dtype=torch.complex128, device=dev)
    ppa_ms = [0.0, 0.0]
    ppa_launches = 0
    if args.ppa:
        from synth import HA_EV
        ppa_w = ppa_real_freqs(args.ppa)
        ppa_eta = PPA_ETA_EV / HA_EV
        wt_d = torch.empty((ng, ng), dtype=torch.complex128, device=dev)
        pr_d = torch.empty_like(wt_d)
        model_d = torch.empty((args.ppa, ng, ng), dtype=torch.complex128, device=dev)
        # one event triple per timed step, read after the timed region
        ppa_ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]

    ppa_done = []

    def ppa_step(timed):
        ev = ppa_ev[len(ppa_done)] if timed else None
        if ev:
            ev[0].record(stream)
        lib.ppa_fit(inv_d[0], inv_d[1], PPA_OMEGA_P, wt_d, pr_d, stream.cuda_stream)
        if ev:
            ev[1].record(stream)
        lib.ppa_eval(wt_d, pr_d, ppa_w, ppa_eta, model_d, stream.cuda_stream)
        if ev:
            ev[2].record(stream)
            ppa_done.append(ev)

    def step(timed=False):
        ctx.compute_rho(0)
        ctx.build_invert(0, inv_d)
        if args.ppa:
            ppa_step(timed)

    for _ in range(args.warmup):
        step()
    ctx.synchronize()
    nt = ctx.get_transitions().shape[0]
    groups = ctx.pole_groups() if args.grouping else None
    ctx.get_stats()  # reset the stage timers
    _, _, _, l0 = ctx.get_stats()

    def barrier():
        if dist is not None:
            dist.barrier()

    barrier()
    torch.cuda.synchronize(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step(timed=True)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
    barrier()
    for a, b, c in ppa_done:
        ppa_ms[0] += a.elapsed_time(b)
        ppa_ms[1] += b.elapsed_time(c)
        ppa_launches += 1 + -(-args.ppa // 32)
    ms_total = ev0.elapsed_time(ev1)
    ctx.synchronize()
    st_ms, st_bytes, st_flops, l1 = ctx.get_stats()
    launches = (l1 - l0) + ppa_launches
    ms_total = max_over_ranks(ms_total, dist, dev)
    ms_step = ms_total / args.steps
    flops_step = chi0_flops(ng, nt, nw)
    value = whole_job_tflops(world, flops_step, ms_step)

    # ---- end to end: host buffers, copies inside the timed region
    pin_gv = [torch.from_numpy(np.ascontiguousarray(s.gvec[ik, :s.npw[ik]])).pin_memory() for ik in range(s.nk)]
    pin_cf = [torch.from_numpy(np.ascontiguousarray(s.coef[ik, :, :s.npw[ik]])).pin_memory() for ik in range(s.nk)]
    out_h = torch.empty((args.ppa or nw, ng, ng), dtype=torch.complex128).pin_memory()
    h2d = sum(int(x.numel() * x.element_size()) for x in pin_gv + pin_cf) + 2 * s.eps.nbytes
    d2h = int(out_h.numel() * out_h.element_size())

    # host wall time of each call of an end-to-end step (the calls return as
    # soon as their work is queued, except the last, which copies the result
    # to the host and waits for it)
    phase_ms = {"set_wavefunctions": 0.0, "set_energies": 0.0, "compute_rho": 0.0, "build_invert_and_copy": 0.0}

    def e2e_step():
        t = [time.perf_counter()]
        for ik in range(s.nk):
            ctx.set_wavefunctions(ik, pin_gv[ik], pin_cf[ik])
        t.append(time.perf_counter())
        ctx.set_energies(s.eps, s.occ)
        t.append(time.perf_counter())
        ctx.compute_rho(0)
        t.append(time.perf_counter())
        if args.ppa:
            ctx.build_invert(0, inv_d)
            ppa_step(False)
            out_h.copy_(model_d)     # the model on the real axis, device -> host
        else:
            ctx.build_invert(0, out_h)   # device -> host copy of the result, synchronises
        t.append(time.perf_counter())
        for k, a, b in zip(phase_ms, t[:-1], t[1:]):
            phase_ms[k] += (b - a) * 1e3

    e2e_clk = None
    if args.no_e2e:
        e2e_ms = None
    else:
        e2e_step()
        for k in phase_ms:
            phase_ms[k] = 0.0
        e2e_steps = max(1, min(args.steps, 3))
        barrier()
        torch.cuda.synchronize(dev)
        with ClockSampler(local) as e2e_clk:
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                e2e_step()
            torch.cuda.synchronize(dev)
            barrier()
            e2e_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps
        e2e_ms = max_over_ranks(e2e_ms, dist, dev)
        phase_ms = {k: v / e2e_steps for k, v in phase_ms.items()}
    # data for the error against the oracle: one more step with chi0 kept
    cmp_data = None
    if jobs is not None:
        jobs.start_chi0()
        chi_d = torch.empty_like(inv_d)
        ctx.compute_rho(0)
        ctx.build_invert(0, inv_d, chi_d)
        torch.cuda.synchronize(dev)
        two = [0, nw - 1]
        cmp_data = {"chi_sub": chi_d[:, :ERR_G, :ERR_G].cpu().numpy(),
                    "chi_two": chi_d[two].cpu().numpy(), "inv_two": inv_d[two].cpu().numpy(), "two": two}
        for m in cmp_data["chi_two"]:
            jobs.start_gj(m)
        del chi_d
    sigma_line = None
    if args.sigma:
        # the self-energy kernel I (Eq. I_c) on the real-axis eps~^-1 of this
        # step: the plasmon-pole model's matrices, or the direct real-axis ones
        lo, hi = args.sigma
        src = model_d if args.ppa else inv_d
        nws, nqp = int(src.shape[0]), hi - lo
        out_s = torch.empty((nws, s.nk, s.nb, nqp, nqp), dtype=torch.complex128, device=dev)
        ctx.build_sigma_i(0, lo, hi, src, out_s)   # plans the buffers
        ctx.synchronize()
        ctx.get_stats()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.sigma_steps):
            ctx.build_sigma_i(0, lo, hi, src, out_s)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        sig_ms = e0.elapsed_time(e1) / args.sigma_steps
        sms, _, _, _ = ctx.get_stats()
        sms = {k: v / args.sigma_steps for k, v in sms.items()}
        T = s.nk * s.nb * nqp
        n_i, n_j = -(-ng // 64), -(-T // 64)
        alg = 8.0 * ng * ng * T * nws                     # complex N_G^2 T multiply-adds per frequency
        issued = 3 * 2 * 128 * 128 * (-(-ng // 64) * 64) * n_i * n_j * nws
        ybytes = n_i * n_j * 4096 * (8.0 if args.precision == "mixed" else 16.0) * nws   # Y tiles read by the dot
        sigma_line = {"window": [lo, hi], "n_freqs": nws, "n_transitions": T, "ms_per_call": sig_ms,
                      "stage_ms_per_call": {"rho": sms["rho"], "split": sms["weights"],
                                            "contract": sms["contract"], "dot": sms["reduce"]},
                      "contract_tflops": alg / (sms["contract"] * 1e-3) / 1e12,
                      "contract_issued_tflops": issued / (sms["contract"] * 1e-3) / 1e12,
                      "dot_y_gbs": ybytes / (sms["reduce"] * 1e-3) / 1e9}
    ctx.get_stats()
    ctx.close()
    fp64_line = fp64_form(args, lib, s, nt, stream, dev) if compare else None
    base_line = None
    if jobs is not None:
        base_line = baseline_and_error(s, nt, jobs, cmp_data, fp64_line)

    if rank != 0:
        return
    pk = peaks()
    # dominant kernel: the stage with the largest device time (events on the
    # stream each stage's kernels are launched on)
    dom = max(st_ms, key=lambda k: st_ms[k])
    per_step_ms = {k: v / args.steps for k, v in st_ms.items()}
    roofs = dict(STAGE_ROOF)
    if args.precision == "fp64":  # every stage on the FP64 units
        roofs.update({"contract": ("fp64", "TFLOP/s", "k_chi0_fp64"), "rho": ("fp64", "TFLOP/s", "k_rho_pairs"),
                      "wf_grid": ("fp64", "TFLOP/s", "k_wf_to_mixed")})
    bound, unit, kname = roofs[dom]
    # (complex weights of real frequencies: the same kernel over every tile)
    extra = {}
    if unit == "GB/s":
        achieved = st_bytes[dom] / (per_step_ms[dom] * 1e-3) / 1e9
        peak, psrc = pk["hbm_gbs"], f"HBM copy ({pk['source']})"
    elif bound == "tensor":
        # algorithmic Hermitian count (4 N_G (N_G + 1) N_T per frequency) over
        # the contraction time; beside it the tensor pipe's share of the BF16
        # products actually issued (3 per k-step over the lower-triangle tiles)
        achieved = st_flops[dom] / (per_step_ms[dom] * 1e-3) / 1e12
        peak, psrc = pk["bf16_tflops_sustained"], f"BF16 dense sustained ({pk['source']})"
        mpad = -(-2 * ng // 256) * 256
        kpad = -(-nt // 64) * 64
        nI, nJ = mpad // 128, mpad // 256
        # an imaginary frequency is one Hermitian contraction (128 x 256
        # tiles covering the lower triangle), a real one one contraction with
        # complex weights (every 128 x 128 tile)
        if args.real_axis:
            issued = 3 * 2 * 128 * 128 * nI * nI * kpad * nw
        else:
            issued = 3 * 2 * 128 * 256 * (nI * nJ - nJ * (nJ - 1)) * kpad * nw
        extra = {"issued_tflops": issued / (per_step_ms[dom] * 1e-3) / 1e12,
                 "issued_frac": issued / (per_step_ms[dom] * 1e-3) / 1e12 / peak}
    elif bound == "fp64":
        achieved = st_flops[dom] / (per_step_ms[dom] * 1e-3) / 1e12
        peak, psrc = FP64_PEAK, FP64_SRC
    else:
        achieved = st_flops[dom] / (per_step_ms[dom] * 1e-3) / 1e12
        peak, psrc = FP32_PEAK, FP32_SRC
    traffic, tsrc = stored_traffic(kname, workload_tag(args))
    roof = {"kernel": kname, "stage": dom, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "peak_source": psrc, "traffic": traffic, "traffic_source": tsrc}
    roof.update(extra)
    stages = stage_rooflines(args, st_ms, st_bytes, st_flops, pk, nt, ng, nw)
    ppa_line = None
    if args.ppa:
        n2 = ng * ng
        fit_bytes = 64.0 * n2
        eval_bytes = (32.0 * -(-args.ppa // 32) + 16.0 * args.ppa) * n2
        fit_ms, eval_ms = ppa_ms[0] / args.steps, ppa_ms[1] / args.steps
        ppa_line = {"omega_p_ha": PPA_OMEGA_P, "n_real_freqs": args.ppa, "fit_ms": fit_ms, "eval_ms": eval_ms,
                    "fit_gbs": fit_bytes / (fit_ms * 1e-3) / 1e9, "eval_gbs": eval_bytes / (eval_ms * 1e-3) / 1e9,
                    "fit_hbm_frac": fit_bytes / (fit_ms * 1e-3) / 1e9 / pk["hbm_gbs"],
                    "eval_hbm_frac": eval_bytes / (eval_ms * 1e-3) / 1e9 / pk["hbm_gbs"],
                    "bytes_per_element": {"fit": 64, "eval": eval_bytes / n2},
                    # the evaluation is bound by the FP64 units: 20 FP64 operations per
                    # element and frequency (the reciprocal counted as one)
                    "eval_fp64_tflops": 20.0 * n2 * args.ppa / (eval_ms * 1e-3) / 1e12,
                    "eval_fp64_frac": 20.0 * n2 * args.ppa / (eval_ms * 1e-3) / 1e12 / FP64_PEAK,
                    "fp64_peak_source": FP64_SRC}
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": ("bf16x3/fp32 (chi0), fp32 (rho), f64 (eps^-1)" if args.precision == "mixed" else "f64"), "data": "synthetic",
        "config": {"workload": workload_name(args), "n_transitions": nt, "l2": "inputs larger than L2 (mixed grids 32 GB, rho 12 GB)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "stage_ms_per_step": per_step_ms,
        "roofline": roof,
        "stage_roofline": stages,
        "e2e": (None if e2e_ms is None else
                {"value": whole_job_tflops(world, flops_step, e2e_ms), "unit": "TFLOP/s", "ms_per_step": e2e_ms,
                 "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                 "phase_host_ms_per_step": phase_ms,
                 # the e2e steps follow the timed region: the SM clock they ran at
                 "clocks": e2e_clk.summary() if e2e_clk is not None else None}),
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    if ppa_line is not None:
        line["ppa"] = ppa_line
    if groups is not None:
        line["pole_groups"] = {"threshold_ha": args.grouping, "groups": groups[0],
                               "grouped_contraction": groups[1]}
    if sigma_line is not None:
        sg = sigma_line
        sg["contract_issued_frac"] = sg["contract_issued_tflops"] / pk["bf16_tflops_sustained"]
        sg["contract_peak_source"] = f"BF16 dense sustained ({pk['source']})"
        sg["dot_y_hbm_frac"] = sg["dot_y_gbs"] / pk["hbm_gbs"]
        line["sigma"] = sg
    if fp64_line is not None:
        f = {k: v for k, v in fp64_line.items() if not k.startswith("_")}
        f["speedup_vs_fp64_form_measured"] = f["ms_per_step"] / f["mixed_ms_per_step"]
        f["speedup_vs_fp64_form_derived_at_nw"] = f["derived_ms_at_nw"] / ms_step
        line["fp64_form"] = f
    if base_line is not None:
        line["cpu_baseline"], line["error"] = base_line
    elif fp64_line is not None:
        line["error"] = {"eps_inv_mixed_vs_fp64_form": fp64_line["_eps_vs_fp64"]}
    if not args.no_cpu_baseline and base_line is None:
        import oracle as O
        G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], s.ng)
        nks = 4
        dt, fl = oracle_sample(s, nks, G)
        line["cpu_baseline"] = {"value": fl / dt / 1e12, "unit": "TFLOP/s", "cores": cpu_cores(), "kind": "oracle",
                                "sample": f"FP64 numpy oracle, all {nks * 2944} transitions of {nks} of {s.nk} "
                                          f"k points, all {s.ng} G and {s.freqs.size} frequencies",
                                "seconds": dt}
    print(json.dumps(line), flush=True)


def fp64_form(args, lib, s, nt, stream, dev):
    """The plain FP64 form of the same step on the first FP64_NW frequencies
    (one step, timed by CUDA events on the stream its kernels run on), and the
    mixed form on the same frequencies for the equal-work ratio.  The derived
    FP64 time for all frequencies is the measured one with its
    frequency-dependent stages scaled linearly (stated as derived)."""
    import dataclasses
    import torch
    nwf = min(args.fp64_nw, s.freqs.size)
    s2 = dataclasses.replace(s, freqs=s.freqs[:nwf])
    ng = s.ng

    def run(prec, steps, warm):
        ctx = lib.Chi0.for_system(s2, precision=prec, stream=stream.cuda_stream)
        gv = [torch.from_numpy(np.ascontiguousarray(s2.gvec[ik, :s2.npw[ik]])).to(dev) for ik in range(s2.nk)]
        cf = [torch.from_numpy(np.ascontiguousarray(s2.coef[ik, :, :s2.npw[ik]])).to(dev) for ik in range(s2.nk)]
        for ik in range(s2.nk):
            ctx.set_wavefunctions(ik, gv[ik], cf[ik])
        ctx.set_energies(s2.eps, s2.occ)
        del gv, cf
        inv = torch.empty((nwf, ng, ng), dtype=torch.complex128, device=dev)
        chi = torch.empty_like(inv)
        for _ in range(warm):
            ctx.compute_rho(0)
            ctx.build_invert(0, inv, chi)
        ctx.synchronize()
        ctx.get_stats()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            ctx.compute_rho(0)
            ctx.build_invert(0, inv, chi)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        sms, _, _, _ = ctx.get_stats()
        out = (ms, {k: v / steps for k, v in sms.items()}, chi[:, :ERR_G, :ERR_G].cpu().numpy(), inv.cpu().numpy())
        ctx.close()
        del inv, chi
        torch.cuda.empty_cache()
        return out

    mixed_ms, _, _, inv_mixed = run(lib.CHI0_MIXED_BF16X3, 2, 1)
    with ClockSampler(int(dev.index or 0)) as clk:
        f_ms, f_stage, f_chi_sub, inv_f = run(lib.CHI0_FP64, 1, 0)
    freq_ms = f_stage["weights"] + f_stage["contract"] + f_stage["reduce"] + f_stage["dyson"]
    derived = f_ms + freq_ms * (s.freqs.size / nwf - 1.0)
    return {"frequencies": nwf, "ms_per_step": f_ms, "stage_ms_per_step": f_stage,
            "mixed_ms_per_step": mixed_ms, "ms_per_frequency": freq_ms / nwf,
            "derived_ms_at_nw": derived,
            "derived_note": f"measured at {nwf} frequencies; the frequency-dependent stages scaled to "
                            f"{s.freqs.size} (derived, not measured)",
            "tflops": chi0_flops(ng, nt, nwf) / (f_ms * 1e-3) / 1e12,
            "mixed_tflops": chi0_flops(ng, nt, nwf) / (mixed_ms * 1e-3) / 1e12, "clocks": clk.summary(),
            "_chi_sub": f_chi_sub,
            "_eps_vs_fp64": {"frequencies": list(range(nwf)),
                             "values": [rel_fro(inv_mixed[i], inv_f[i]) for i in range(nwf)],
                             "note": "mixed-form eps~^-1 against the plain FP64 form's (full N_G)"}}


def baseline_and_error(s, nt, jobs, cmp_data, fp64_line):
    """The CPU baseline leg's results: its time (the baseline) and the errors
    of the GPU path against it."""
    ref, t_oracle = jobs.chi0()
    gj = jobs.gj_results()
    jobs.close()
    nw = s.freqs.size
    per_w = [rel_fro(cmp_data["chi_sub"][i], ref[i]) for i in range(nw)]
    err = {
        "what": "relative Frobenius error ||X - X_oracle||_F / ||X_oracle||_F per frequency",
        "chi0_subblock": {"g_indices": f"0..{ERR_G - 1}", "max": max(per_w), "median": float(np.median(per_w)),
                          "per_frequency": per_w, "tolerance": 1e-5},
        "eps_inv_dyson_vs_oracle_gauss_jordan": {
            "frequencies": cmp_data["two"],
            "values": [rel_fro(cmp_data["inv_two"][j], gj[j]) for j in range(len(gj))],
            "note": "the GPU's eps~^-1 at full N_G against the oracle's Gauss-Jordan inversion of eps~ "
                    "built from the GPU's own chi0 (isolates the Dyson step)"},
    }
    if fp64_line is not None:
        nwf = fp64_line["frequencies"]
        err["chi0_subblock_fp64_form"] = [rel_fro(fp64_line["_chi_sub"][i], ref[i]) for i in range(nwf)]
        err["eps_inv_mixed_vs_fp64_form"] = fp64_line["_eps_vs_fp64"]
    flops = chi0_flops(ERR_G, nt, nw)
    base = {"value": flops / t_oracle / 1e12, "unit": "TFLOP/s", "cores": jobs.nproc, "kind": "oracle",
            "sample": f"FP64 numpy oracle, the G_0..G_{ERR_G - 1} sub-block of chi0 over all {nt} transitions and "
                      f"{nw} frequencies (rho by direct convolution for those G), k points split over "
                      f"{jobs.nproc} worker processes; TFLOP/s of the 4 N_G (N_G + 1) N_T N_w count at N_G = {ERR_G}",
            "seconds": t_oracle}
    return base, err


def large_states_device(spec, dev):
    """The states of the large workload generated on the device, k point by k
    point, by the recipe of synth.make_system: complex Gaussian draws keyed by
    (seed, k) (torch's Philox generator on the GPU instead of numpy's PCG64),
    orthonormalised per k by QR (cuSOLVER through torch.linalg.qr, FP32), the
    time-reversal partner -k derived by conjugation, c_{k'}(G) =
    conj(c_k(-G - G1)), and self-partner k points orthonormalised in real
    coordinates so that c(G) = conj(c(-G - 2k)) holds exactly.  Yields
    (ik, gvec [npw][3] int32, coef [nbands][npw] complex64), both on dev."""
    import math
    import torch
    from synth import kgrid_fractions, sphere_miller, tr_partner
    kgrid = tuple(int(v) for v in spec.kgrid)
    nk = kgrid[0] * kgrid[1] * kgrid[2]
    nb = spec.n_bands
    kfrac = kgrid_fractions(kgrid)
    gen = torch.Generator(device=dev)
    done = np.zeros(nk, dtype=bool)

    def sphere(ik):
        g = sphere_miller(kfrac[ik], spec.a, spec.kc)
        return g, torch.from_numpy(np.ascontiguousarray(g)).to(dev)

    for ik in range(nk):
        if done[ik]:
            continue
        jk = tr_partner(ik, kgrid)
        g, g_d = sphere(ik)
        gen.manual_seed(spec.seed * 1000003 + ik)
        if jk == ik:
            two_k = np.rint(2.0 * kfrac[ik]).astype(np.int64)
            where = {tuple(v): p for p, v in enumerate(g.tolist())}
            partner = np.array([where[tuple((-v - two_k).tolist())] for v in g.astype(np.int64)])
            idx = np.arange(g.shape[0])
            fixed = np.nonzero(partner == idx)[0]
            reps = np.nonzero(partner > idx)[0]
            nf, nr = fixed.size, reps.size
            x = torch.randn((nf + 2 * nr, nb), generator=gen, device=dev, dtype=torch.float32)
            q = torch.linalg.qr(x, mode="reduced")[0]
            c = torch.zeros((nb, g.shape[0]), dtype=torch.complex64, device=dev)
            s2 = 1.0 / math.sqrt(2.0)
            xr, yr = q[nf:nf + nr].T, q[nf + nr:].T
            c[:, torch.from_numpy(fixed).to(dev)] = q[:nf].T.to(torch.complex64)
            c[:, torch.from_numpy(reps).to(dev)] = torch.complex(s2 * xr, s2 * yr)
            c[:, torch.from_numpy(partner[reps]).to(dev)] = torch.complex(s2 * xr, -s2 * yr)
            done[ik] = True
            yield ik, g_d, c
            continue
        z = torch.randn((g.shape[0], nb), generator=gen, device=dev, dtype=torch.complex64)
        c = torch.linalg.qr(z, mode="reduced")[0].T.contiguous()
        yield ik, g_d, c
        g1 = np.rint(kfrac[ik] + kfrac[jk]).astype(np.int64)
        gp, gp_d = sphere(jk)
        where = {tuple(v): p for p, v in enumerate(g.tolist())}
        src = np.array([where[tuple((-v - g1).tolist())] for v in gp.astype(np.int64)], dtype=np.int64)
        yield jk, gp_d, c[:, torch.from_numpy(src).to(dev)].conj().contiguous()
        done[ik] = done[jk] = True


def run_large(args, rank, world, dist):
    """The large workload (12x12x12 k, 24 + 976 bands, ~4000 PW, FFT 72^3,
    N_G = 3000, 64 imaginary frequencies) at one q point: the transitions
    (40.5 million; rho alone would be 971 GB) streamed in band blocks through
    rho, the operand split and the contraction, chi0 summed in FP64, then the
    FP64 Dyson step.  One step is the whole q point; it runs in minutes, so
    the warm-up is a step of a smaller k grid of the same system shape."""
    import dataclasses
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_1902_03837_gb300 import chi0 as lib
    from synth import cfg_large, large_energies, sphere_miller, kgrid_fractions
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    spec = cfg_large(kgrid=tuple(args.kgrid) if args.kgrid else (12, 12, 12), nw=args.nw if args.nw != 32 else 64)
    iq = args.large_iq
    spec = dataclasses.replace(spec, q_frac=(spec.q_frac[iq],))

    def make_ctx(sp):
        kf = kgrid_fractions(sp.kgrid)
        npw_max = max(sphere_miller(kf[k], sp.a, sp.kc).shape[0] for k in range(kf.shape[0]))
        ctx = lib.Chi0(a=sp.a, kgrid=sp.kgrid, nbands=sp.n_bands, npw_max=npw_max, fft=sp.fft, ng=sp.ng,
                       q_frac=np.array(sp.q_frac), omega=np.array(sp.freqs), eta=sp.eta,
                       spin_factor=sp.spin_factor, precision=lib.CHI0_MIXED_BF16X3, stream=stream.cuda_stream)
        t0 = time.perf_counter()
        npw = []
        for ik, gv, cf in large_states_device(sp, dev):
            ctx.set_wavefunctions(ik, gv, cf)
            npw.append(int(gv.shape[0]))
        eps = large_energies(sp)
        occ = np.zeros_like(eps)
        occ[:, :sp.n_occ] = 1.0
        ctx.set_energies(eps, occ)
        ctx.synchronize()
        ctx.set_band_blocks(args.large_bands, args.large_kblock)
        return ctx, time.perf_counter() - t0, npw_max, float(np.mean(npw))

    ng, nw = spec.ng, len(spec.freqs)
    inv = torch.empty((nw, ng, ng), dtype=torch.complex128, device=dev)
    # warm-up: the same shape on a 2x2x2 k grid (kernels, plans, clocks)
    wctx, _, _, _ = make_ctx(dataclasses.replace(spec, kgrid=(2, 2, 2), q_frac=((0.5, 0.0, 0.0),)))
    for _ in range(max(1, args.warmup)):
        wctx.compute_rho(0)
        wctx.build_invert(0, inv)
    wctx.synchronize()
    wctx.close()
    torch.cuda.empty_cache()
    ctx, gen_s, npw_max, npw_mean = make_ctx(spec)
    ctx.get_stats()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            ctx.compute_rho(0)
            ctx.build_invert(0, inv)
        e1.record(stream)
        torch.cuda.synchronize(dev)
    ctx.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, dev)
    st_ms, st_bytes, st_flops, launches = ctx.get_stats()
    nt = int(ctx.get_transitions().shape[0])
    spectrum = torch.linalg.eigvalsh(inv[[0, nw - 1]]).cpu().numpy()
    ctx.close()
    if rank != 0:
        return
    pk = peaks()
    flops = chi0_flops(ng, nt, nw)
    per = {k: v / args.steps for k, v in st_ms.items()}
    cargs = argparse.Namespace(precision="mixed", steps=args.steps)
    stages = stage_rooflines(cargs, st_ms, st_bytes, st_flops, pk, nt, ng, nw)
    con = stages.get("contract", {})
    line = {
        "metric": METRIC, "value": whole_job_tflops(world, flops, ms), "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x3/fp32 (chi0), fp32 (rho), f64 (eps^-1)", "data": "synthetic",
        "config": {"workload": f"large: a=10 bohr, k {'x'.join(map(str, spec.kgrid))}, 24+976 bands, ~4000 PW "
                               f"(mean {npw_mean:.0f}, max {npw_max}), FFT 72^3, N_G=3000, {nw} imaginary GL "
                               f"frequencies in [0,100] eV, q = ({spec.q_frac[0][0]:.4f},0,0), complex64",
                   "n_transitions": nt, "band_blocks": [args.large_bands, args.large_kblock],
                   "l2": "inputs larger than L2", "warmup_note": "warm-up steps on a 2x2x2 k grid of the same shape",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "input_generation_s": gen_s, "stage_ms_per_step": per, "stage_roofline": stages,
        "roofline": {"kernel": "k_herk_wide", "stage": "contract", "bound": "tensor",
                     "achieved": con.get("tflops"), "peak": pk["bf16_tflops_sustained"], "unit": "TFLOP/s",
                     "frac": con.get("tensor_frac"), "peak_source": f"BF16 dense sustained ({pk['source']})",
                     "traffic": None, "traffic_source": "not captured for this workload"},
        "eps_inv_spectrum_w0_wlast": [float(spectrum.min()), float(spectrum.max())],
        "gpu_launches": int(launches), "clocks": clk.summary(), "e2e": None,
    }
    print(json.dumps(line), flush=True)


def run_terminator(args, rank, world, dist):
    """The learned-terminator workload: systems of 6x6x6 k, 12 occupied bands,
    ~1500 PW, FFT 32^3, N_G = 500, 16 imaginary frequencies, q = (1/6,0,0),
    each with 800 bands (the full-band sum, the reference) and its first 100
    (truncated).  The network is trained on the GPU by the library's kernels
    on the pairs of the training systems (seeds 4000...) and judged on the
    held-out ones (seeds 5000...) against the full-band sum, beside the
    truncated sum alone and the Bruneval-Gonze extrapolar correction."""
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_1902_03837_gb300 import chi0 as lib
    from paper_1902_03837_gb300 import terminator as term
    from synth import cfg_learned, large_energies, kgrid_fractions, sphere_miller, HA_EV
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    st = stream.cuda_stream
    nb_t = args.term_truncated
    spec0 = cfg_learned()
    kf = kgrid_fractions(spec0.kgrid)
    npw_max = max(sphere_miller(kf[k], spec0.a, spec0.kc).shape[0] for k in range(kf.shape[0]))

    def ctx_for(nb):
        return lib.Chi0(a=spec0.a, kgrid=spec0.kgrid, nbands=nb, npw_max=npw_max, fft=spec0.fft, ng=spec0.ng,
                        q_frac=np.array(spec0.q_frac), omega=np.array(spec0.freqs), eta=spec0.eta,
                        spin_factor=spec0.spin_factor, precision=lib.CHI0_MIXED_BF16X3, stream=st)

    ctx_f, ctx_t = ctx_for(spec0.n_bands), ctx_for(nb_t)
    nw, ng = len(spec0.freqs), spec0.ng
    chi_f = torch.empty((nw, ng, ng), dtype=torch.complex128, device=dev)
    chi_t = torch.empty_like(chi_f)

    def load(seed, truncated):
        """The system's states into the full-band context and the truncated ones."""
        spec = cfg_learned(seed=seed)
        for ik, gv, cf in large_states_device(spec, dev):
            ctx_f.set_wavefunctions(ik, gv, cf)
            ct = cf[:nb_t].contiguous()
            for c in truncated:
                c.set_wavefunctions(ik, gv, ct)
        eps = large_energies(spec)
        occ = np.zeros_like(eps)
        occ[:, :spec.n_occ] = 1.0
        ctx_f.set_energies(eps, occ)
        for c in truncated:
            c.set_energies(np.ascontiguousarray(eps[:, :nb_t]), np.ascontiguousarray(occ[:, :nb_t]))
        return eps

    t0 = time.perf_counter()
    X, T = [], []
    gpu_ms = 0.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for seed in range(4000, 4000 + args.term_train):
        load(seed, [ctx_t])
        e0.record(stream)
        for c, out in ((ctx_f, chi_f), (ctx_t, chi_t)):
            c.compute_rho(0)
            c.build_chi0(0, out)
        e1.record(stream)
        n = chi_t.numel()
        x = torch.empty((n, 5), dtype=torch.float32, device=dev)
        t = torch.empty((n, 2), dtype=torch.float32, device=dev)
        ctx_t.term_features(0, chi_t, x, chi_f, t)
        torch.cuda.synchronize(dev)
        gpu_ms += e0.elapsed_time(e1)
        X.append(x)
        T.append(t)
    X = torch.cat(X)
    T = torch.cat(T)
    t_data = time.perf_counter() - t0
    e0.record(stream)
    params, hist = term.train(X, T, steps=args.term_steps, batch=4096, lr=2e-3, seed=1, stream=st,
                              log_every=max(1, args.term_steps // 10))
    e1.record(stream)
    torch.cuda.synchronize(dev)
    train_ms = e0.elapsed_time(e1)
    del X, T
    torch.cuda.empty_cache()
    # held-out systems: truncated, truncated + network, truncated + extrapolar correction
    ctx_c = ctx_for(nb_t)
    ctx_c.set_terminator(params, True)
    ctx_b = ctx_for(nb_t)
    chi_c = torch.empty_like(chi_f)
    errs = {"truncated": [], "truncated_plus_network": [], "truncated_plus_bg_1.5Ha": [],
            "truncated_plus_bg_mean_omitted": []}
    for seed in range(5000, 5000 + args.term_test):
        eps = load(seed, [ctx_t, ctx_c, ctx_b])
        for c, out in ((ctx_f, chi_f), (ctx_t, chi_t), (ctx_c, chi_c)):
            c.compute_rho(0)
            c.build_chi0(0, out)
        nf = torch.linalg.norm(chi_f).item()
        errs["truncated"].append(torch.linalg.norm(chi_t - chi_f).item() / nf)
        errs["truncated_plus_network"].append(torch.linalg.norm(chi_c - chi_f).item() / nf)
        for key, eb in (("truncated_plus_bg_1.5Ha", 1.5), ("truncated_plus_bg_mean_omitted",
                                                             float(eps[:, nb_t:].mean()))):
            ctx_b.set_bg_terminator(eb)
            ctx_b.compute_rho(0)
            ctx_b.build_chi0(0, chi_c)
            errs[key].append(torch.linalg.norm(chi_c - chi_f).item() / nf)
        ctx_b.set_bg_terminator(1.5, on=False)
    for c in (ctx_f, ctx_t, ctx_c, ctx_b):
        c.synchronize()
        c.close()
    if rank != 0:
        return
    summary = {k: {"mean": float(np.mean(v)), "std": float(np.std(v)), "max": float(np.max(v))}
               for k, v in errs.items()}
    line = {
        "metric": "learned band-sum terminator: held-out relative Frobenius error of chi0 against the full-band sum",
        "value": summary["truncated_plus_network"]["mean"], "unit": "relative error", "higher_is_better": False,
        "n_gpus": world, "steps": args.term_steps, "warmup": 0, "dtype": "bf16 network, bf16x3/fp32 chi0",
        "data": "synthetic", "vs_baseline": None, "scaling": "weak",
        "config": {"workload": f"learned terminator: 6x6x6 k, 12 occupied, {nb_t} of 800 bands, ~1500 PW, FFT 32^3, "
                               f"N_G=500, 16 imaginary GL frequencies, q=(1/6,0,0); {args.term_train} training "
                               f"systems (seeds 4000..), {args.term_test} held-out (seeds 5000..)",
                   "network": "5 -> 128 -> 128 -> 2 tanh, BF16 operands, FP32 accumulation, Adam lr 2e-3, "
                              f"batch 4096, {args.term_steps} steps"},
        "held_out_error": summary, "held_out_per_system": errs,
        "loss_history": hist, "data_seconds": t_data, "chi0_pairs_gpu_ms": gpu_ms, "train_ms": train_ms,
    }
    print(json.dumps(line), flush=True)


def run_batching(args, rank, world, dist):
    """The batching workload: 16 seeded metallic systems of different sizes,
    every q point of each (4-20 per system, 200 problems), all in one batch
    (one persistent rho launch, every other kernel in one CUDA graph; the q
    points of a system share its mixed grids), against the same problems one
    at a time, and the first problem in the plain FP64 form."""
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_1902_03837_gb300 import chi0 as lib
    from synth import make_batching_system
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    st = stream.cuda_stream
    systems = [make_batching_system(s_, nq_max=args.batch_nq) for s_ in range(args.batch_systems)]
    probs = [(si, iq) for si, sy in enumerate(systems) for iq in range(sy.q_frac.shape[0])]
    outs = [torch.empty((systems[si].freqs.size, systems[si].ng, systems[si].ng), dtype=torch.complex128,
                        device=dev) for si, _ in probs]
    ctxs = []
    for sy in systems:
        c = lib.Chi0.for_system(sy, precision=lib.CHI0_MIXED_BF16X3, stream=st, occ_drop_tol=1e-12)
        c.load_system(sy)
        ctxs.append(c)
    t0 = time.perf_counter()
    batch = lib.Batch([ctxs[si] for si, _ in probs], [iq for _, iq in probs], outs, nstreams=args.batch_streams)
    create_s = time.perf_counter() - t0
    streams_of, tuned_ms = batch.info()
    width = batch.rho_width()
    for _ in range(args.warmup):
        batch.run(st)
    batch.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    with ClockSampler(local) as clk:
        ev[0].record(stream)
        for _ in range(args.steps):
            batch.run(st)
        ev[1].record(stream)
        torch.cuda.synchronize(dev)
    batch.synchronize()
    batch_ms = max_over_ranks(ev[0].elapsed_time(ev[1]) / args.steps, dist, dev)
    keep = outs[0].clone()
    batch.close()
    for c in ctxs:
        c.close()
    torch.cuda.empty_cache()
    # the same problems one at a time, each system in a context of its own
    # (device time of compute_rho + build_invert per problem, after one
    # untimed pass over the system's q points)
    per_problem = [0.0] * len(probs)
    nts = [0] * len(probs)
    pe = [torch.cuda.Event(enable_timing=True) for _ in range(2 * len(probs))]
    for si, sy in enumerate(systems):
        c = lib.Chi0.for_system(sy, precision=lib.CHI0_MIXED_BF16X3, stream=st, occ_drop_tol=1e-12)
        c.load_system(sy)
        mine = [k for k, (sj, _) in enumerate(probs) if sj == si]
        for k in mine:
            c.compute_rho(probs[k][1])
            nts[k] = int(c.get_transitions().shape[0])
            c.build_invert(probs[k][1], outs[k])
        torch.cuda.synchronize(dev)
        for k in mine:
            pe[2 * k].record(stream)
            c.compute_rho(probs[k][1])
            c.build_invert(probs[k][1], outs[k])
            pe[2 * k + 1].record(stream)
        torch.cuda.synchronize(dev)
        for k in mine:
            per_problem[k] = pe[2 * k].elapsed_time(pe[2 * k + 1])
        c.synchronize()
        c.close()
        torch.cuda.empty_cache()
    seq_ms = sum(per_problem)
    diff0 = ((outs[0] - keep).abs().pow(2).sum() / keep.abs().pow(2).sum()).sqrt().item()
    flops = sum(chi0_flops(systems[si].ng, nts[k], systems[si].freqs.size) for k, (si, _) in enumerate(probs))
    # the plain FP64 form of the first problem, for the speedup at the same size
    s0 = systems[0]
    c64 = lib.Chi0.for_system(s0, precision=lib.CHI0_FP64, stream=st, occ_drop_tol=1e-12)
    c64.load_system(s0)
    o64 = torch.empty_like(outs[0])
    c64.compute_rho(0)
    c64.build_invert(0, o64)
    torch.cuda.synchronize(dev)
    ev[0].record(stream)
    c64.compute_rho(0)
    c64.build_invert(0, o64)
    ev[1].record(stream)
    torch.cuda.synchronize(dev)
    fp64_ms = ev[0].elapsed_time(ev[1])
    err0 = ((o64 - keep).abs().pow(2).sum() / o64.abs().pow(2).sum()).sqrt().item()
    c64.close()
    if rank != 0:
        return
    nq = [int(sy.q_frac.shape[0]) for sy in systems]
    line = {
        "metric": "batched chi0(q,w) + eps^-1 throughput (algorithmic Hermitian TFLOP/s)",
        "value": whole_job_tflops(world, flops, batch_ms), "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": batch_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3/fp32 (chi0), fp32 (rho), f64 (eps^-1)",
        "data": "synthetic",
        "config": {"workload": f"batching: {len(systems)} metallic systems (seeds 3000-{3000 + len(systems) - 1}; "
                               "a 8-14 bohr, 4x4x4 k, 64 bands, 400-4000 PW, N_G 200-1500, 8-64 imaginary GL "
                               "frequencies, Fermi-Dirac 0.05 eV), every q point of each",
                   "problems": len(probs), "q_points_per_system": nq,
                   "ng": [sy.ng for sy in systems], "nw": [int(sy.freqs.size) for sy in systems],
                   "n_transitions_total": int(sum(nts)), "helper_streams": args.batch_streams,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "batch_ms": batch_ms, "one_at_a_time_ms": seq_ms, "speedup_vs_one_at_a_time": seq_ms / batch_ms,
        "batch_create_s": create_s, "rho_width": width, "tuned_contraction_ms": tuned_ms,
        "problems_per_stream": [streams_of.count(h) for h in range(args.batch_streams)],
        "batch_vs_one_at_a_time_problem0": diff0,
        "fp64_problem0_ms": fp64_ms, "mixed_problem0_ms": per_problem[0],
        "speedup_vs_fp64_problem0": fp64_ms / per_problem[0], "error_vs_fp64_problem0": err0,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kgrid", type=lambda v: tuple(int(x) for x in v.split(",")), default=None,
                    help="smaller k grid for profiling runs, e.g. 4,2,2 (default 8,8,8)")
    ap.add_argument("--nw", type=int, default=32, help="number of imaginary frequencies")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"],
                    help="mixed: FP32 rho, BF16x3 tensor-core chi0, FP64 Dyson (default); "
                         "fp64: the plain FP64 form of every step, for the speedup comparison")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end (host buffer) measurement")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the plain FP64 form and the error against the oracle")
    ap.add_argument("--fp64-nw", type=int, default=2, help="frequencies of the plain FP64 form's timed step")
    ap.add_argument("--real-axis", action="store_true",
                    help="real frequencies on (0, 100] eV with 0.1 eV broadening (two contractions each, "
                         "general Dyson step)")
    ap.add_argument("--bg-terminator", type=float, default=None, metavar="EV",
                    help="apply the Bruneval-Gonze extrapolar correction with this extrapolar energy (eV)")
    ap.add_argument("--ppa", type=int, default=0, metavar="NW",
                    help="plasmon-pole path: chi0 and eps^-1 at w = 0 and i 1 Ha only, the Godby-Needs fit and "
                         "the model on NW real frequencies on (0, 100] eV")
    ap.add_argument("--sigma", type=lambda v: tuple(int(x) for x in v.split(",")), default=None,
                    metavar="LO,HI", help="then time the self-energy kernel I (Eq. I_c) for the bands [LO, HI) at k "
                                          "on the real-axis eps~^-1 of --ppa or --real-axis")
    ap.add_argument("--sigma-steps", type=int, default=2)
    ap.add_argument("--batching", action="store_true",
                    help="the batching workload (16 metallic systems, every q point) in one batch, against one at a time")
    ap.add_argument("--batch-systems", type=int, default=16, help="systems of the batching workload (from the first)")
    ap.add_argument("--batch-nq", type=int, default=None, help="keep only the first NQ q points of each system")
    ap.add_argument("--batch-streams", type=int, default=4, help="helper streams of the batch")
    ap.add_argument("--flat-bands", action="store_true",
                    help="dispersionless bands: every k has the band energies of k = 0 (degenerate poles)")
    ap.add_argument("--grouping", type=float, default=0.0, metavar="HA",
                    help="degenerate-pole grouping threshold (Ha); large groups use the grouped contraction")
    ap.add_argument("--terminator", action="store_true",
                    help="the learned-terminator workload: train on chi0 pairs, report the held-out error")
    ap.add_argument("--term-train", type=int, default=200, help="training systems of the terminator workload")
    ap.add_argument("--term-test", type=int, default=50, help="held-out systems of the terminator workload")
    ap.add_argument("--term-steps", type=int, default=20000, help="Adam steps of the terminator training")
    ap.add_argument("--term-truncated", type=int, default=100, help="bands of the truncated sum")
    ap.add_argument("--workload", default="precision", choices=["precision", "large"],
                    help="large: 12x12x12 k, 1000 bands, N_G 3000, 64 frequencies, one q point, band-block streamed")
    ap.add_argument("--large-iq", type=int, default=0, help="q point (0..7) of the large workload")
    ap.add_argument("--large-bands", type=int, default=122, help="n bands per block (large workload)")
    ap.add_argument("--large-kblock", type=int, default=64, help="k points per block (large workload)")
    args = ap.parse_args()
    if args.ppa and (args.real_axis or args.ppa < 0):
        ap.error("--ppa takes a positive count and excludes --real-axis")
    if args.sigma and not (args.ppa or args.real_axis):
        ap.error("--sigma needs real-axis frequencies: --ppa NW or --real-axis")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
        dist = tdist
    if args.batching:
        run_batching(args, rank, world, dist)
    elif args.workload == "large":
        run_large(args, rank, world, dist)
    elif args.terminator:
        run_terminator(args, rank, world, dist)
    else:
        run_ours(args, rank, world, dist)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
