"""Benchmark: compact FMG (Algorithm 3) DoF/s to discretization error on GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload NAME]

A step is one whole compact FMG solve (L = 1 .. L_max, N IR iterations per
level) of the workload with its right-hand side already on the device.  Under
torchrun each rank solves its own replica (weak scaling; the method has no
exchange step across replicas).  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "compact-FMG DoF/s to discretization error"

WORKLOADS = {
    # name: (problem generator, L_max, description)
    "poisson3d_2049": ("poisson3d_manufactured", 11,
                       "3-D Poisson 2049^3 grid (2047^3 = 8.58e9 interior DoF), zero Dirichlet, "
                       "RHS matrix-free from u=sin(pi x)sin(pi y)sin(pi z)(1+x^2yz)"),
    "poisson3d_513": ("poisson3d_manufactured", 9,
                      "3-D Poisson 513^3 grid (511^3 = 1.33e8 DoF), same RHS as poisson3d_2049"),
    "diffusion3d_1025": ("diffusion3d_grf", 10,
                         "3-D -div(k grad u) = 1, 1025^3 grid (1023^3 = 1.07e9 DoF), k = exp(g), g a seeded "
                         "Gaussian random field (sigma 1, correlation length 0.1, 256 Fourier features), "
                         "binary32 cycle inside FP64 iterative refinement"),
    "adjoint3d_257": ("diffusion3d_grf", 8,
                      "3-D adjoint: J = |u - u_obs|^2 / 2 for -div(exp(m) grad u) = 1 on 257^3, m a seeded "
                      "GRF (sigma 0.5, seed 2), u_obs from m + GRF (sigma 0.1, seed 3); a step is the forward "
                      "compact FMG, J, and the backward (adjoint compact FMG + gradient kernel) through "
                      "torch.autograd"),
    "diffusion3d_513": ("diffusion3d_grf", 9,
                        "3-D -div(k grad u) = 1, 513^3 grid (511^3 = 1.33e8 DoF), k = exp(g) as diffusion3d_1025"),
    "diffusion3d_257": ("diffusion3d_grf", 8,
                        "3-D -div(k grad u) = 1, 257^3 grid, k = exp(g) as diffusion3d_1025"),
    "poisson3d_257": ("poisson3d_fourier", 8,
                      "3-D Poisson 257^3 grid (255^3 DoF), RHS = 8 seeded Fourier modes"),
    "poisson2d_257": ("poisson2d_manufactured", 8,
                      "2-D Poisson 257^2 grid, u=sin(pi x)sin(pi y)(1+x^2 y)"),
}
DEFAULT_WORKLOAD = "poisson3d_2049"
# cycle arithmetic: exact (int64), binary32 or binary64 V-cycle inside the exact refinement
ARITH_NAMES = ["exact", "fp32", "fp64"]
DTYPE_NAMES = ["int64", "f32 cycle + int64 refinement", "f64 cycle + int64 refinement"]


def source_sha() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2511_19036_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def read_profile(kernel: str, workload: str, key: str):
    """A per-unit figure (``key``) of ``kernel`` from the committed ncu summary, if it
    was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "%s_%s.md" % (kernel, workload))
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m_sha = re.search(r"source_sha:\s*([0-9a-f]+)", txt)
    m_val = re.search(r"%s:\s*([0-9.eE+-]+)" % re.escape(key), txt)
    if not m_sha or not m_val or m_sha.group(1) != source_sha():
        return None
    return float(m_val.group(1))


def read_traffic(kernel: str, workload: str):
    return read_profile(kernel, workload, "dram_bytes_per_dof")


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_fmg_rate(prob_name: str, L: int, cfg, max_seconds: float = 30.0):
    """Time the CPU oracle's compact FMG on the same problem at level L.
    Returns (DoF/s, seconds, dofs)."""
    import cmg_problems
    import oracle
    prob = cmg_problems.make_problem(prob_name, L)
    o = oracle.Oracle.for_problem(prob, b1=cfg.b1, b2=cfg.b2, N=cfg.N_ir, nu1=cfg.nu1, nu2=cfg.nu2,
                                  omega=cfg.omega, arith=cfg.arith, smoother=cfg.smoother)
    t0 = time.perf_counter()
    o.fmg()
    dt = time.perf_counter() - t0
    dofs = ((1 << L) - 1) ** prob.dim
    return dofs / dt, dt, dofs


def oracle_rate_one_thread(prob_name: str, L: int, cfg):
    """The oracle's compact FMG on one host thread (a child process, since the
    OpenMP thread count is fixed at start). Returns (DoF/s, seconds, dofs) or None."""
    import subprocess
    code = ("import json, sys; sys.path.insert(0, %r); import bench, oracle; oracle.build(); "
            "from paper_2511_19036_gb300.cmg_config import config_for; "
            "cfg = config_for(%r, %d, arith=%d, smoother=%d); "
            "print(json.dumps(bench.oracle_fmg_rate(%r, %d, cfg)))"
            % (ROOT, prob_name, cfg.L_max, cfg.arith, cfg.smoother, prob_name, L))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        return None
    return tuple(json.loads(r.stdout.strip().splitlines()[-1]))


class gpu_local_cpus:
    """Runs the block on the CPUs next to the GPU (its sysfs local_cpulist), so
    that host buffers pinned inside it land in the GPU's NUMA node; the thread's
    affinity is restored afterwards.  No-op where the list is not available."""

    def __init__(self, device: int):
        self.device = device
        self.old = None

    def __enter__(self):
        try:
            import torch
            p = torch.cuda.get_device_properties(self.device)
            path = "/sys/bus/pci/devices/%04x:%02x:%02x.0/local_cpulist" % (
                p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
            cpus = set()
            for part in open(path).read().strip().split(","):
                if "-" in part:
                    lo, hi = part.split("-")
                    cpus.update(range(int(lo), int(hi) + 1))
                elif part:
                    cpus.add(int(part))
            if cpus:
                self.old = os.sched_getaffinity(0)
                os.sched_setaffinity(0, cpus)
        except (OSError, ValueError, AttributeError):
            self.old = None
        return self

    def __exit__(self, *exc):
        if self.old is not None:
            os.sched_setaffinity(0, self.old)
        return False


def max_over_ranks(x: float, dist, device: str) -> float:
    """The job's time is the slowest rank's (x on one rank; all ranks get it)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, dofs_per_rank: int, seconds: float) -> float:
    """Whole-job DoF/s: every rank solves its own replica of dofs_per_rank unknowns
    (weak scaling), all of them within `seconds` (the maximum over ranks)."""
    return world * dofs_per_rank / seconds


def smoother_of(args, prob_name: str) -> int:
    # red-black Gauss-Seidel is built for the Poisson problem
    return 1 if args.smoother == "rbgs" and not prob_name.startswith("diffusion") else 0


def cycle_name(cfg) -> str:
    return "V(%d,%d) %s" % (cfg.nu1, cfg.nu2, "red-black Gauss-Seidel" if cfg.smoother else "weighted Jacobi")


def pick_sample_level(prob_name: str, Lmax: int, dim: int) -> int:
    # bounded oracle sample: a few to about 10 s of host work per solve on a
    # 16-core host (3-D L = 9 is 1.3e8 DoF)
    if prob_name.startswith("diffusion"):  # the coefficient field is drawn on the host here
        return min(Lmax, 7 if dim == 3 else 10)
    return min(Lmax, 9 if dim == 3 else 12)


def run_reference(args, wl):
    prob_name, Lmax, desc = WORKLOADS[wl]
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count()))
    import oracle
    oracle.build()
    from paper_2511_19036_gb300.cmg_config import config_for
    cfg = config_for(prob_name, Lmax, arith=ARITH_NAMES.index(args.arith),
                     smoother=smoother_of(args, prob_name))
    dim = cfg.dim
    Ls = pick_sample_level(prob_name, Lmax, dim)
    for _ in range(args.warmup):
        oracle_fmg_rate(prob_name, max(2, Ls - 2), cfg)
    rates, times = [], []
    for _ in range(args.steps):
        r, dt, dofs = oracle_fmg_rate(prob_name, Ls, cfg)
        rates.append(r)
        times.append(dt)
    value = statistics.median(rates)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count()))
    sample = "oracle compact FMG of the same problem at L_max=%d (%d DoF) per step" % (Ls, dofs)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl, "description": desc, "dim": dim, "L_max": Lmax, "b1": cfg.b1,
                   "b2": cfg.b2, "N_ir": cfg.N_ir, "cycle": cycle_name(cfg), "omega": cfg.omega},
        "cpu_baseline": {"value": value, "unit": "DoF/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "DoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_gpu(args, wl):
    import numpy as np
    import torch

    import cmg_problems
    from paper_2511_19036_gb300 import _build
    _build.build()
    from paper_2511_19036_gb300 import cmg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    prob_name, Lmax, desc = WORKLOADS[wl]
    prob = cmg_problems.make_problem(prob_name, Lmax, seed=rank)
    cfg = cmg.config_for(prob_name, Lmax, arith=ARITH_NAMES.index(args.arith),
                         smoother=smoother_of(args, prob_name))
    diffusion = bool(getattr(prob, "coef", 0))
    stream = torch.cuda.Stream()
    # events around the finest-level launches only (the roofline kernel); the solve
    # runs as a CUDA graph after the first two warm-up solves
    solver = cmg.Solver(cfg, stream=stream, timing="top")
    solver.set_rhs(prob.tables, prob.scale_exp)
    if diffusion:  # the seeded coefficient field, drawn on the device (input data)
        kfield = prob.kfield(device="cuda").reshape(-1).contiguous()
        torch.cuda.synchronize()
        solver.set_coefficient(kfield)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        solver.fmg_solve()
    barrier()
    clk = ClockSampler(local)
    clk.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reports = []
    ev0.record(stream)
    for _ in range(args.steps):
        reports.append(solver.fmg_solve())
    ev1.record(stream)
    barrier()
    clocks = clk.stop()
    ms_total = max_over_ranks(ev0.elapsed_time(ev1), dist, "cuda")
    ms_step = ms_total / args.steps
    dofs = reports[0]["dofs"]
    value = job_rate(world, dofs, ms_step * 1e-3)

    # dominant kernel: the finest-level Jacobi sweep (events on the solver's stream)
    sw_ms = sum(r["sweep_ms_total"] for r in reports)
    sw_n = sum(r["sweep_launches"] for r in reports)
    # a diffusion sweep also reads the nodal binary32 coefficient once per launch
    # (4 B per node); the library's byte model counts sections and temporaries only
    coef_bytes = 4.0 * ((1 << Lmax) + 1) ** cfg.dim if diffusion else 0.0
    sw_bytes = sum(r["sweep_alg_bytes"] for r in reports) + sw_n * coef_bytes
    peak, peak_kind = measured_peak_hbm()
    achieved = (sw_bytes / sw_n) / (sw_ms / sw_n * 1e-3) / 1e9 if sw_n and sw_ms > 0 else None
    # the finest-level sweep kernel: the specialised 3-D red / black half-sweeps on
    # the exact red-black path, else the generic (or floating-point) sweep
    sweep_kernel = ("k_sweep_fp" if cfg.arith else
                    "k_fast_sweep" if (cfg.smoother and cfg.dim == 3) else "k_sweep")
    prof_wl = wl + ("_rbgs" if cfg.smoother else "_jacobi")
    traffic_per_dof = read_traffic(sweep_kernel, prof_wl)
    roofline = {"kernel": "%s<%d> finest level" % (sweep_kernel, cfg.dim),
                "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None,
                "traffic": traffic_per_dof * dofs if traffic_per_dof else None,
                "alg_bytes_per_launch": sw_bytes / sw_n if sw_n else None,
                "coefficient_bytes_per_launch": coef_bytes,
                "avg_launch_ms": sw_ms / sw_n if sw_n else None,
                "peak_kind": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind}
    # the same launches against the survey's algorithmic bytes (bits per finest DoF of
    # mantissas, exponent bytes and the coarse sources each launch must touch once):
    # red-black: red = r + z-source + y~ written, black = y~ + r + z-source + u~ read and
    # written; Jacobi: down = 3 y~/r sections, up = the same + z-source, last up = 2
    # sections + z-source + u~ read and written.  z-source = (b2 + 1.25)/8 + 1.
    sec_r, sec_u = cfg.b2 + 0.25, cfg.b1 + 0.25
    zsrc = (cfg.b2 + 1.25) / 8 + 1
    if cfg.smoother:
        survey_bits = ((2 * sec_r + zsrc) + (2 * sec_r + zsrc + 2 * sec_u)) / 2
    else:
        survey_bits = (3 * sec_r + (3 * sec_r + zsrc) + (2 * sec_r + zsrc + 2 * sec_u)) / 3
    if achieved:
        roofline["survey_bytes_per_dof"] = survey_bits / 8
        ach_s = survey_bits / 8 * dofs / (sw_ms / sw_n * 1e-3) / 1e9
        roofline["achieved_survey"] = ach_s
        roofline["frac_survey"] = ach_s / peak
    # the bound that holds: instruction issue (4 warp-instructions per SM and clock)
    # with the ncu instruction count per 32-value row of the same kernels
    inst_row = read_profile(sweep_kernel, prof_wl, "warp_inst_per_row")
    issue = None
    if inst_row and sw_n and sw_ms > 0:
        nsm = torch.cuda.get_device_properties(local).multi_processor_count
        mhz = (clocks or {}).get("sm_mhz") or (clocks or {}).get("sm_max_mhz")
        rows = int(cmg.lib().cmg_section_blocks(cfg.dim, Lmax))
        ach = inst_row * rows / (sw_ms / sw_n * 1e-3)
        pk = 4.0 * nsm * mhz * 1e6 if mhz else None
        issue = {"kernel": roofline["kernel"], "unit": "warp-instructions/s", "achieved": ach, "peak": pk,
                 "frac": ach / pk if pk else None, "warp_inst_per_row": inst_row,
                 "peak_kind": "4 issue slots per SM per clock x %d SMs x %s MHz (sampled SM clock)" % (nsm, mhz)}
    whole_frac = (reports[0]["alg_bytes"] / (ms_step * 1e-3) / 1e9) / peak
    # Sec. 6.1.4 storage model for this workload (mantissa bits, CMG vs BFPMG) next to
    # the measured layout (exponents, row padding and the Jacobi ping-pong included)
    smod = cmg.storage_model(cfg.dim, Lmax, cfg.k_u, cfg.k_r, cfg.b1, cfg.b2)
    storage = {"cmg_fmg_bits_per_dof": smod["cmg_fmg_bits"] / smod["dofs"],
               "bfpmg_fmg_bits_per_dof": smod["bfpmg_fmg_bits"] / smod["dofs"],
               "fmg_saving": smod["fmg_saving"], "vector_saving": smod["vector_saving"],
               "measured_bits_per_dof": reports[0]["persistent_bits"] / dofs}
    # end to end through the public API: H2D of the step's inputs (the RHS tables,
    # from pinned memory) and D2H of the step's result (the compact solution).
    with gpu_local_cpus(local):
        tab_pinned = torch.from_numpy(np.ascontiguousarray(prob.tables)).pin_memory()
    nb = [int(cmg.lib().cmg_section_blocks(cfg.dim, l)) for l in range(1, Lmax + 1)]
    Wu = [cfg.k_u * (Lmax - l) + cfg.b1 for l in range(1, Lmax + 1)]
    with gpu_local_cpus(local):
        out_w = [torch.empty(nb[i] * Wu[i], dtype=torch.int32).pin_memory() for i in range(Lmax)]
        out_e = [torch.empty(nb[i], dtype=torch.int8).pin_memory() for i in range(Lmax)]
    h2d = tab_pinned.numel() * 4
    d2h = sum(w.numel() * 4 + e.numel() for w, e in zip(out_w, out_e))
    e2e_times, phases = [], []
    lib = cmg.lib()
    for it in range(max(1, min(args.steps, 3))):
        barrier()
        t0 = time.perf_counter()
        st = lib.cmg_set_rhs_separable(solver._h, prob.nterms, tab_pinned.data_ptr(), prob.scale_exp)
        assert st == 0
        t1 = time.perf_counter()
        solver.fmg_solve()
        t2 = time.perf_counter()
        for l in range(1, Lmax + 1):
            st = lib.cmg_get_section(solver._h, 0, l, out_w[l - 1].data_ptr(), out_e[l - 1].data_ptr())
            assert st == 0
        barrier()
        t3 = time.perf_counter()
        e2e_times.append(t3 - t0)
        phases.append((t1 - t0, t2 - t1, t3 - t2))
    e2e_s = max_over_ranks(statistics.median(e2e_times), dist, "cuda")
    graph_stats = solver.graph_stats()

    # where one solve spends its device time, per kernel kind: one more solve with
    # events around every launch, after the timed region
    solver.set_timing(True)
    solver.fmg_solve()
    kernels = {k: {"ms": round(v["ms"], 4), "launches": v["launches"],
                   "GB_per_s": round(v["bytes"] / (v["ms"] * 1e-3) / 1e9, 1) if v["ms"] > 0 else None}
               for k, v in solver.kernel_stats().items() if v["launches"]}

    # discretization-error check on sampled planes of the decoded solution
    n = (1 << Lmax) - 1
    h = 2.0 ** -Lmax
    planes = [n // 4, n // 2, (3 * n) // 4] if cfg.dim == 3 else [0]
    errs, norms = [], []
    x = (np.arange(n) + 1.0) * h
    nodal_rel = None
    if not diffusion:
        for z in planes:
            u = solver.decode_solution(z, 1).cpu().numpy()[0]
            Y, X = np.meshgrid(x, x, indexing="ij")
            ue = prob.exact_u(X, Y, (z + 1) * h) if cfg.dim == 3 else prob.exact_u(X, Y)
            errs.append(float(np.max(np.abs(u - ue))))
            norms.append(float(np.max(np.abs(ue))))
        nodal_rel = max(errs) / max(norms)
    # diffusion (no closed form): the solution against a reference solve of the
    # same discrete problem with the binary64 cycle, wider widths and more IR
    # iterations (the FP64 reference on the GPU), on sampled planes
    def sampled_diff(sa, sb):
        dmax, umax = 0.0, 0.0
        for z in planes:
            a = sa.decode_solution(z, 1).cpu().numpy()[0]
            b = sb.decode_solution(z, 1).cpu().numpy()[0]
            dmax = max(dmax, float(np.max(np.abs(a - b))))
            umax = max(umax, float(np.max(np.abs(b))))
        return dmax / umax

    diffusion_vs_reference, fp32_vs_fp64 = None, None
    if diffusion:
        import dataclasses
        rcfg = dataclasses.replace(cfg, b1=14, b2=10, N_ir=16, arith=2)
        ref = cmg.Solver(rcfg, stream=stream)
        ref.set_rhs(prob.tables, prob.scale_exp)
        ref.set_coefficient(kfield)
        ref.fmg_solve()
        diffusion_vs_reference = {"max_rel_diff_sampled": sampled_diff(solver, ref),
                                  "reference": "b1=14, b2=10, N_ir=16, binary64 cycle"}
        # the other floating-point cycle at the same widths, solved once after the
        # timed region (device time by CUDA events on the solver's stream)
        if not args.no_compare:
            ocfg = dataclasses.replace(cfg, arith=1 if cfg.arith == 2 else 2)
            other = cmg.Solver(ocfg, stream=stream, timing=True)
            other.set_rhs(prob.tables, prob.scale_exp)
            other.set_coefficient(kfield)
            other_ms = other.fmg_solve()["solve_ms"]
            mine = {"cycle_ms": ms_step, "rel_err_vs_reference": diffusion_vs_reference["max_rel_diff_sampled"]}
            theirs = {"cycle_ms": other_ms, "rel_err_vs_reference": sampled_diff(other, ref)}
            f32, f64 = (mine, theirs) if cfg.arith == 1 else (theirs, mine)
            fp32_vs_fp64 = {"fp32_cycle_ms": f32["cycle_ms"], "fp64_cycle_ms": f64["cycle_ms"],
                            "max_rel_diff_sampled": sampled_diff(other, solver),
                            "rel_err_fp32_cycle_vs_reference": f32["rel_err_vs_reference"],
                            "rel_err_fp64_cycle_vs_reference": f64["rel_err_vs_reference"],
                            "note": "the same widths and IR; one solve of the other form after the timed region"}
            del other
        del ref
    # Sec. 7.1 at this size: the H1 error of the solution against that of a
    # near-lossless solve of the same discrete problem (Jacobi V(2,2), b1 = b2 = 12,
    # N = 8), integrated on the GPU slab by slab (manufactured 3-D problems)
    discretization_check = None
    if args.h1 and not diffusion and cfg.dim == 3 and prob_name.endswith("manufactured"):
        import dataclasses
        from cmg_problems.diagnostics import h1_error_slabs
        rcfg = dataclasses.replace(cmg.config_for(prob_name, Lmax), b1=min(12, 32 - cfg.k_u * (Lmax - 1)),
                                   b2=12, N_ir=8)
        ref = cmg.Solver(rcfg, stream=stream)
        ref.set_rhs(prob.tables, prob.scale_exp)
        ref.fmg_solve()
        e_ref = h1_error_slabs(prob, lambda z0, nz: ref.decode_solution(z0, nz), Lmax)
        del ref
        e_cmg = h1_error_slabs(prob, lambda z0, nz: solver.decode_solution(z0, nz), Lmax)
        discretization_check = {"h1_error": e_cmg, "h1_error_reference": e_ref, "ratio": e_cmg / e_ref,
                                "criterion": "Sec. 7.1: ratio <= 2", "met": e_cmg <= 2 * e_ref,
                                "reference": "Jacobi V(2,2), b1=%d, b2=12, N_ir=8" % rcfg.b1}
    # the precision split (binary32 cycle inside the exact refinement) against the
    # exact cycle and the plain binary64 cycle, on the same GPU and problem, after
    # the timed region: each other form is solved once (its device time by CUDA
    # events on the solver's stream) and compared on the sampled planes
    fp32_vs_exact, precision_forms = None, None
    if not diffusion and not args.no_compare:
        precision_forms = {ARITH_NAMES[cfg.arith]: {"cycle_ms": ms_step, "nodal_rel_err_sampled": nodal_rel,
                                                    "max_rel_diff_vs_timed_sampled": 0.0}}
        for ar in (0, 1, 2):
            if ar == cfg.arith:
                continue
            other = cmg.config_for(prob_name, Lmax, arith=ar, smoother=cfg.smoother)
            if cmg.params_check(other) != cmg.OK:
                continue
            ref = cmg.Solver(other, stream=stream)
            ref.set_rhs(prob.tables, prob.scale_exp)
            ref_ms = ref.fmg_solve()["solve_ms"]
            dmax, umax, err_other = 0.0, 0.0, []
            for z in planes:
                a = solver.decode_solution(z, 1).cpu().numpy()[0]
                b = ref.decode_solution(z, 1).cpu().numpy()[0]
                Y, X = np.meshgrid(x, x, indexing="ij")
                ue = prob.exact_u(X, Y, (z + 1) * h) if cfg.dim == 3 else prob.exact_u(X, Y)
                dmax = max(dmax, float(np.max(np.abs(a - b))))
                umax = max(umax, float(np.max(np.abs(a))))
                err_other.append(float(np.max(np.abs(b - ue))))
            precision_forms[ARITH_NAMES[ar]] = {"cycle_ms": ref_ms, "nodal_rel_err_sampled": max(err_other) / max(norms),
                                                "max_rel_diff_vs_timed_sampled": dmax / umax}
            del ref
        if "exact" in precision_forms and "fp32" in precision_forms:
            ex, f3 = precision_forms["exact"], precision_forms["fp32"]
            fp32_vs_exact = {"max_rel_diff_sampled": max(ex["max_rel_diff_vs_timed_sampled"],
                                                         f3["max_rel_diff_vs_timed_sampled"]),
                             "exact_cycle_ms": ex["cycle_ms"], "fp32_cycle_ms": f3["cycle_ms"],
                             "nodal_rel_err_exact_cycle": ex["nodal_rel_err_sampled"],
                             "nodal_rel_err_fp32_cycle": f3["nodal_rel_err_sampled"],
                             "note": "one solve of the other form after the timed region"}

    # the finest level's coarse sources formed on the fly (cmg_set_two_level): the
    # same exact solve without the int64 w and u^ of level L_max - 1, once after
    # the timed region, against the timed (materialized) one
    two_level = None
    if cfg.arith == 0 and not diffusion and Lmax >= 3 and not args.no_compare:
        tsol = cmg.Solver(cfg, stream=stream, two_level=True)
        tsol.set_rhs(prob.tables, prob.scale_exp)
        trep = tsol.fmg_solve()
        same = all(np.array_equal(solver.decode_solution(z, 1).cpu().numpy(), tsol.decode_solution(z, 1).cpu().numpy())
                   for z in planes)
        two_level = {"cycle_ms": trep["solve_ms"], "temp_bytes_per_dof": trep["temp_bytes"] / dofs,
                     "temp_bytes_per_dof_materialized": reports[0]["temp_bytes"] / dofs,
                     "same_solution_sampled": bool(same),
                     "note": "one solve on the two-level path after the timed region"}
        del tsol

    if rank != 0:
        return 0
    # CPU oracle baseline on a bounded sample of the same problem (rank 0, N = 1)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count()))
        import oracle
        oracle.build()
        Ls = pick_sample_level(prob_name, Lmax, cfg.dim)
        r, dt, sdofs = oracle_fmg_rate(prob_name, Ls, cfg)
        cpu = {"value": r, "unit": "DoF/s", "cores": int(os.environ["OMP_NUM_THREADS"]), "kind": "oracle",
               "sample": "oracle compact FMG of the same problem at L_max=%d (%d DoF), %.1f s" % (Ls, sdofs, dt)}
        if not diffusion:
            one = oracle_rate_one_thread(prob_name, min(Ls, 7 if cfg.dim == 3 else 10), cfg)
            if one:
                cpu["single_core"] = {"value": one[0], "unit": "DoF/s", "cores": 1,
                                      "sample": "the same at %d DoF, %.1f s" % (one[2], one[1])}
    launches = int(sum(r["launches"] for r in reports))
    if diffusion:  # a diffusion restriction step is two kernels, counted once by the library
        launches += args.steps * sum(kernels.get(k, {}).get("launches", 0) for k in ("restrict_top", "restrict_lower"))
    line = {
        "metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE_NAMES[cfg.arith],
        "data": "synthetic",
        "config": {"workload": wl, "description": desc, "dim": cfg.dim, "L_max": Lmax, "dofs": dofs,
                   "b1": cfg.b1, "b2": cfg.b2, "N_ir": cfg.N_ir, "cycle": cycle_name(cfg),
                   "omega": cfg.omega, "arith": ARITH_NAMES[cfg.arith] + (" cycle" if cfg.arith else ""),
                   "l2": "working set larger than L2" if dofs > 1e8 else
                   "working set fits L2 (state per step re-read from L2)",
                   "parallelism": "replicas x%d" % world},
        "bits_per_dof": reports[0]["persistent_bits"] / dofs,
        "temp_bytes_per_dof": reports[0]["temp_bytes"] / dofs,
        # the problem's inputs held on the device: the separable right-hand-side
        # tables, and for diffusion the binary32 nodal coefficient (boundary included)
        "input_bytes_per_dof": {"rhs_tables": prob.tables.size * 4 / dofs,
                                "coefficient": (((1 << Lmax) + 1) ** cfg.dim * 4 / dofs) if diffusion else 0.0},
        "alg_bytes_per_step": reports[0]["alg_bytes"],
        "whole_solve_hbm_frac": whole_frac,
        "nodal_rel_err_sampled": nodal_rel,
        "discretization_check": discretization_check,
        "fp32_vs_exact": fp32_vs_exact,
        "precision_forms": precision_forms,
        "diffusion_vs_reference": diffusion_vs_reference,
        "fp32_vs_fp64": fp32_vs_fp64,
        "two_level": two_level,
        "roofline": roofline,
        "issue_roofline": issue,
        "fast_kernels": solver.fast_stats(),
        "kernels_one_solve": kernels,
        "solve_graph": dict(graph_stats, note="solves run as one CUDA graph launch (timed and end-to-end "
                            "steps after two warm-up solves)"),
        "storage_model": storage,
        "cpu_baseline": cpu,
        "e2e": {"value": job_rate(world, dofs, e2e_s), "unit": "DoF/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "phases_ms": [[round(1e3 * x, 2) for x in p] for p in phases]},  # set_rhs, solve, D2H
        "gpu_launches": launches,
        "clocks": clocks,
    }
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_adjoint(args, wl):
    """The adjoint workload: DoF/s of one gradient evaluation (forward + backward)."""
    import numpy as np
    import torch

    from cmg_problems.diffusion import diffusion_grf
    from paper_2511_19036_gb300 import _build
    _build.build()
    from paper_2511_19036_gb300 import cmg
    from paper_2511_19036_gb300.adjoint import diffusion_solve

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    _, Lmax, desc = WORKLOADS[wl]
    dim = 3
    prob = diffusion_grf(dim, Lmax, seed=2 + 10 * rank, sigma=0.5)
    pert = diffusion_grf(dim, Lmax, seed=3 + 10 * rank, sigma=0.1)
    m = prob.g_field("cuda")
    k = torch.exp(m).to(torch.float32).reshape(-1).contiguous()
    k_obs = torch.exp(m + pert.g_field("cuda")).to(torch.float32).reshape(-1).contiguous()
    n = (1 << Lmax) - 1
    dofs = n ** dim
    cfg = cmg.config_for("diffusion3d_grf", Lmax)
    with gpu_local_cpus(local):
        g_host = torch.ones(dofs, dtype=torch.float64).pin_memory()
    g = g_host.cuda()
    with torch.no_grad():
        u_obs = diffusion_solve(k_obs, g, cfg).reshape(-1)

    def step(c=cfg):
        kt = k.clone().requires_grad_(True)
        gt = g.clone().requires_grad_(True)
        u = diffusion_solve(kt, gt, c).reshape(-1)
        J = 0.5 * torch.sum((u - u_obs) ** 2)
        dk, dg = torch.autograd.grad(J, (kt, gt))
        return J, dk * kt.detach(), dg  # dJ/dm = k dJ/dk for k = exp(m)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()
    clk = ClockSampler(local)
    clk.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        J, dm, dg = step()
    ev1.record()
    barrier()
    clocks = clk.stop()
    ms_step = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, dist, "cuda")
    # end to end: H2D of g, gradient D2H, inside the timed region
    with gpu_local_cpus(local):
        dm_host = torch.empty(dm.numel(), dtype=torch.float32).pin_memory()
    e2e = []
    for _ in range(max(1, min(args.steps, 3))):
        barrier()
        t0 = time.perf_counter()
        g.copy_(g_host, non_blocking=True)
        J, dm, dg = step()
        dm_host.copy_(dm.reshape(-1), non_blocking=True)
        barrier()
        e2e.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(statistics.median(e2e), dist, "cuda")
    # the same gradient with the plain binary64 cycle (same widths and IR), timed
    # once after the timed region, and the difference of the two gradients
    fp32_vs_fp64 = None
    if not args.no_compare:
        import dataclasses
        c64 = dataclasses.replace(cfg, arith=2)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record()
        J64, dm64, dg64 = step(c64)
        e1.record()
        barrier()

        def rel(a, b):
            return float(torch.max(torch.abs(a - b)) / torch.max(torch.abs(b)))
        fp32_vs_fp64 = {"fp32_step_ms": ms_step, "fp64_step_ms": e0.elapsed_time(e1),
                        "rel_diff_J": abs(float(J) - float(J64)) / abs(float(J64)),
                        "max_rel_diff_dJ_dm": rel(dm, dm64), "max_rel_diff_dJ_df": rel(dg, dg64),
                        "note": "forward + adjoint + gradient with the binary64 cycle, once after the timed region"}
    # the dominant kernel, from one timed forward solve of the same problem
    solver = cmg.Solver(cfg, timing=True)
    solver.set_coefficient(k)
    solver.set_rhs_nodal(g)
    rep = solver.fmg_solve()
    peak, peak_kind = measured_peak_hbm()
    kst = solver.kernel_stats()
    ks = kst["sweep_top"]
    nres = kst["restrict_top"]["launches"] + kst["restrict_lower"]["launches"]
    # plus the binary32 coefficient, read once by every finest-level sweep
    coef_bytes = 4.0 * k.numel()
    achieved = (ks["bytes"] + ks["launches"] * coef_bytes) / (ks["ms"] * 1e-3) / 1e9 if ks["ms"] > 0 else None
    if rank != 0:
        return 0
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        Ls = 6
        o_p = diffusion_grf(dim, Ls, seed=2, sigma=0.5)
        ko = o_p.kfield().ravel()
        t0 = time.perf_counter()
        o = oracle.Oracle(dim, Ls, o_p.tables, o_p.scale_exp, b1=cfg.b1, b2=cfg.b2, N=cfg.N_ir, nu1=cfg.nu1,
                          nu2=cfg.nu2, omega=cfg.omega, arith=1, coef=1, kfield=ko)
        o.set_rhs_nodal(np.ones(((1 << Ls) - 1) ** dim))
        o.fmg()
        uo = np.asarray(o.decode_solution()).ravel()
        oa = oracle.Oracle(dim, Ls, o_p.tables, o_p.scale_exp, b1=cfg.b1, b2=cfg.b2, N=cfg.N_ir, nu1=cfg.nu1,
                           nu2=cfg.nu2, omega=cfg.omega, arith=1, coef=1, kfield=ko)
        oa.set_rhs_nodal(np.ldexp(uo, dim * Ls))
        oa.fmg()
        o.gradient_k(uo, np.asarray(oa.decode_solution()).ravel())
        dt = time.perf_counter() - t0
        sd = ((1 << Ls) - 1) ** dim
        cpu = {"value": sd / dt, "unit": "DoF/s", "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count())),
               "kind": "oracle", "sample": "oracle forward + adjoint compact FMG + gradient at L_max=%d (%d DoF), %.1f s"
               % (Ls, sd, dt)}
    line = {
        "metric": "adjoint gradient (forward + adjoint compact FMG + gradient) DoF/s", "value": job_rate(world, dofs, ms_step * 1e-3),
        "unit": "DoF/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 cycle + f64 refinement", "data": "synthetic",
        "config": {"workload": wl, "description": desc, "dim": dim, "L_max": Lmax, "dofs": dofs, "b1": cfg.b1,
                   "b2": cfg.b2, "N_ir": cfg.N_ir, "cycle": cycle_name(cfg),
                   "l2": "working set larger than L2", "parallelism": "replicas x%d" % world},
        "J": float(J.detach()),
        "fp32_vs_fp64": fp32_vs_fp64,
        "roofline": {"kernel": "k_sweep_fp<float, 3> finest level (forward solve)", "bound": "hbm", "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak if achieved else None, "traffic": None,
                     "coefficient_bytes_per_launch": coef_bytes, "peak_kind": peak_kind},
        "cpu_baseline": cpu,
        "e2e": {"value": job_rate(world, dofs, e2e_s), "unit": "DoF/s", "h2d_bytes_per_step": dofs * 8,
                "d2h_bytes_per_step": dm.numel() * 4},
        # forward and adjoint solves (a restriction step is two kernels, counted once by
        # the library) and the gradient kernel
        "gpu_launches": int(2 * (rep["launches"] + nres) + 1),
        "clocks": clocks,
    }
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the solve of the other arithmetic (binary32 cycle / exact cycle)")
    ap.add_argument("--no-h1", dest="h1", action="store_false",
                    help="skip the H1 error check against a near-lossless solve (manufactured 3-D problems)")
    ap.add_argument("--arith", default="exact", choices=["exact", "fp32", "fp64"],
                    help="exact V-cycle, or the binary32 / binary64 V-cycle inside exact iterative refinement")
    ap.add_argument("--smoother", default="rbgs", choices=["rbgs", "jacobi"],
                    help="V(0,1) red-black Gauss-Seidel (Algorithm 1's cycle), or V(2,2) weighted Jacobi; "
                         "diffusion and adjoint workloads always use Jacobi V(2,2)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args, args.workload)
    if args.workload.startswith("adjoint"):
        return run_adjoint(args, args.workload)
    return run_gpu(args, args.workload)


if __name__ == "__main__":
    sys.exit(main())
