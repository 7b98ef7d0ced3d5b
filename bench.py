#!/usr/bin/env python
"""Benchmark: atomic environments per second for the SOAP density expansion and power spectrum on GB300.

A step is one pass of the whole hot path over one batch of synthetic structures: the periodic neighbour list
(rascal_neighbours), the spherical expansion coefficients and the power spectrum (rascal_soap or the separate
calls). The default workload is 512 periodic cubic cells of 64-216 atoms (about 71.7k environments) at
0.05 atoms/A^3 with 4 species, r_cut 5 A, sigma 0.5 A, n_max 12, l_max 9, FP32 coefficients and the packed FP32
power spectrum.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--config batch|...]
Under torchrun each rank processes its own batch (seeded by rank): weak scaling, no data-path collective.
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "atomic environments/sec (expansion+power spectrum, ±gradients) at stated error vs FP64"
UNIT = "env/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
# DRAM bytes (read + written) per environment of the fused pair kernel with the FP32 power spectrum
# (k_expansion<kGramSimt> in its compiled instance for the batch hypers, PACKED layout) on the batch workload's recipe,
# from one ncu capture of a 96-cell case (dram__bytes_read.sum + dram__bytes_write.sum), scaled to a full launch by
# the environments it processes; valid only while that kernel is unchanged, None (reported as null) otherwise. The
# last capture, (7.676 MB + 843.154 MB) / 13 434 environments, is of the kernel before its pair phase indexed the Y
# and G rows by pair position.
FUSED_FP32_TRAFFIC_PER_ENV = None

WORKLOADS = {
    "batch": "512 periodic cubic cells, 64-216 atoms each (uniform), 0.05 atoms/A^3, 4 species uniform, d_min 1.8 A; "
             "r_cut 5 A, sigma 0.5 A, cosine cutoff width 0.5 A, n_max 12, l_max 9; FP32 expansion + FP32 packed "
             "power spectrum",
    "tiny": "1 cubic cell L=10 A, 64 atoms, 1 species; r_cut 5, sigma 0.5, n_max 8, l_max 6",
    "diff": "1 cubic cell, 4096 atoms, 0.05 atoms/A^3, 2 species 1:1; r_cut 5.5, sigma 0.4, n_max 8, l_max 6",
    "large": "1 cubic cell, 32768 atoms, 0.1 atoms/A^3, 3 species 2:1:1, d_min 1.0; r_cut 6, sigma 0.5, n_max 10, l_max 8",
    "mlp": "1 cubic cell, 8192 atoms, 0.06 atoms/A^3, 8 species; r_cut 6, sigma 0.5, n_max 16, l_max 12",
}


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", choices=sorted(WORKLOADS), default="batch")
    ap.add_argument("--layout", choices=["packed", "full"], default="packed")
    ap.add_argument("--ps", choices=["fp32", "bf16", "tf32x3"], default="fp32")
    ap.add_argument("--separate", action="store_true",
                    help="rascal_spherical_expansion + rascal_power_spectrum instead of the fused rascal_soap")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--ref-seconds", type=float, default=150.0,
                    help="host seconds of oracle work that --impl reference spreads over its warm-up and timed steps")
    ap.add_argument("--cpu-seconds", type=float, default=24.0,
                    help="host seconds of oracle work in the CPU baseline, split over its three modes")
    ap.add_argument("--structures", type=int, default=512, help="cells in the batch workload (profiling cases)")
    ap.add_argument("--gradients", action="store_true",
                    help="add the linear energy model and its forces and virial (rascal_linear_energy + rascal_gradients)")
    ap.add_argument("--radial", choices=["spline", "exact", "mlp"], default="spline",
                    help="radial integrals from the FP32 spline, the per-pair FP64 1F1, or the MLP surrogate "
                         "(trained on the GPU before timing)")
    ap.add_argument("--basis", choices=["gto", "dvr"], default="gto",
                    help="radial basis: GTO (Eq. rad-int-gto-1, orthonormalised) or DVR (Eq. rad-int-dvr)")
    ap.add_argument("--gpr", type=int, default=0,
                    help="sparse points per species of a sparse GPR energy model (Eq. sparse-gp) on top of p; 0 = off")
    ap.add_argument("--zeta", type=int, default=2, help="exponent of the GPR polynomial kernel")
    ap.add_argument("--lambda-soap", type=int, default=-1, dest="lambda_soap",
                    help="rank of nu = 2 equivariants computed from c instead of the power spectrum; -1 = off")
    ap.add_argument("--mlp-steps", type=int, default=4000, help="Adam steps of the surrogate's training (setup)")
    ap.add_argument("--select", type=float, default=0.0,
                    help="fraction of the packed power-spectrum features to compute (seeded random selection; "
                         "rascal_soap_selected); 0 = all")
    ap.add_argument("--expansion-only", action="store_true",
                    help="neighbours + coefficients only (rascal_spherical_expansion), no power spectrum")
    ap.add_argument("--cpu-worker", action="store_true", help=argparse.SUPPRESS)
    return ap.parse_args(argv)


def make_system(config: str, rank: int, n_structures: int = 512):
    from synth import structures

    if config == "batch":
        return structures.config_batch(seed=2 + 1000 * rank, n_structures=n_structures)
    fn = {"tiny": structures.config_tiny, "diff": structures.config_diff, "large": structures.config_large,
          "mlp": structures.config_mlp}[config]
    default_seed = {"tiny": 1, "diff": 3, "large": 5, "mlp": 6}[config]
    return fn(seed=default_seed + 1000 * rank)


# ---------------------------------------------------------------------------------------------------- helpers
def load_peaks():
    try:
        with open(PEAKS_FILE) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def load_tensor_peak():
    """Dense BF16 tensor peak (TFLOP/s) measured as a burst, else the fallback figure."""
    try:
        with open(PEAKS_FILE) as fh:
            d = json.load(fh)
        return float(d["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def gpr_setup(args, calc, system, ds, coeffs, ps, sel, rg):
    """A GPR model whose sparse points are the power spectra of seeded atoms of this rank's own workload (one
    untimed soap pass), x_I ~ N(0, 1); returns the model and its config entry with the algorithmic flops of the
    kernel GEMM (2 F sum_s N_s n_s over the centre species)."""
    import numpy as np

    from synth import gpr_sparse_draws

    pairs = calc.neighbours(ds)
    if sel is not None:
        calc.soap_selected(ds, pairs, sel, coeffs=coeffs, ps=ps)
    else:
        calc.soap(ds, pairs, coeffs=coeffs, ps=ps)
    idx, x = gpr_sparse_draws(system.species, calc.species, args.gpr, seed=31)
    import torch

    pm = ps[torch.as_tensor(idx, device=ps.device)].double().cpu().numpy()
    model = rg.GprModel(calc, pm, system.species[idx], x, zeta=args.zeta)
    lab = system.species
    flops = 0.0
    for s in calc.species:
        flops += 2.0 * ps.shape[1] * np.count_nonzero(lab == s) * np.count_nonzero(system.species[idx] == s)
    cfg = {"sparse_per_species": args.gpr, "n_sparse": int(idx.size), "zeta": args.zeta, "features": int(ps.shape[1]),
           "precision": "tf32 operands, fp32 accumulate", "sparse_points": "p of seeded atoms of the workload"}
    return model, {"config": cfg, "flops_energy": flops}


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        smax = max((float(r[2]) for r in rows if r[2].replace(".", "").isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows)}


def dist_init(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _over_ranks(x, device, op):
    import torch

    if not (torch.distributed.is_available() and torch.distributed.is_initialized()) or \
            torch.distributed.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x, device):
    """Largest value over the ranks: the slowest rank sets the job's time. The only collective of a run."""
    import torch

    return _over_ranks(x, device, torch.distributed.ReduceOp.MAX)


def sum_over_ranks(x, device):
    """Sum over the ranks (environments processed by the whole job: each rank has its own batch)."""
    import torch

    return _over_ranks(x, device, torch.distributed.ReduceOp.SUM)


# ---------------------------------------------------------------------------------------------------- CPU oracle
def oracle_step_fn(args, system, h, radial_fn=None):
    """One oracle pass over a list of centres for the workload the flags describe (FP64 numpy); radial_fn, when
    given, replaces the exact radial integrals (the FP64 spline mode)."""
    from oracle import soap as osoap

    w = None
    if args.gradients:
        from synth import linear_weights

        w = linear_weights(h.n_species, h.n_features("packed"), seed=4)
    gpr_model = oracle_gpr_model(args, system, h) if args.gpr else None

    def run(centres):
        if args.lambda_soap >= 0:
            from oracle import lambda_soap as ols

            return ols.equivariants(osoap.spherical_expansion(system, h, centres=centres, radial_fn=radial_fn), h,
                                    args.lambda_soap)
        if gpr_model is not None:
            return oracle_gpr_step(args, system, h, gpr_model, centres, radial_fn)
        if w is not None:  # c, p, adjoint and per-pair gradients of the sampled centres' energy terms
            return osoap.energy_gradients(system, h, w, centres=centres, radial_fn=radial_fn)
        c = osoap.spherical_expansion(system, h, centres=centres, radial_fn=radial_fn)
        return c if args.expansion_only else osoap.power_spectrum(c, h, args.layout)

    return run


_POOL = {}


def _pool_init(argv, system, spline):
    # each process runs one host thread (the environment carries OMP_NUM_THREADS=1 and friends)
    from oracle import soap as osoap

    args = parse_args(argv)
    h = osoap.Hypers(**system.hypers)
    fn = (lambda r, d=False: spline(r, d)) if spline is not None else None
    _POOL["run"] = oracle_step_fn(args, system, h, fn)
    _POOL["run"]([0, 1])  # builds the per-process 1F1 switch points before the timed region


def _pool_task(centres):
    _POOL["run"](centres)
    return len(centres)


def _time_serial(run, order, start, seconds):
    """Grows a sample of centres until one run takes about `seconds`; returns (centres/s, n, seconds, next start)."""
    n = 8
    while True:
        n = int(min(n, len(order) - start))
        t0 = time.perf_counter()
        run(order[start:start + n])
        dt = time.perf_counter() - t0
        start += n
        if dt >= 0.7 * seconds or start >= len(order):
            return n / dt, n, dt, start
        n = int(n * min(8.0, seconds / max(dt, 1e-3)))


def _time_pool(argv, system, spline, order, rate1, procs, seconds):
    """Runs the same oracle pass over a process pool (spawned, one thread each) on a sample sized from the
    single-thread rate; returns (centres/s, n, wall seconds)."""
    import multiprocessing as mp

    import numpy as np

    n = int(min(len(order), max(4 * procs, rate1 * procs * seconds)))
    chunk = max(1, n // (6 * procs))
    tasks = [order[k:k + chunk] for k in range(0, n, chunk)]
    with mp.get_context("spawn").Pool(procs, initializer=_pool_init, initargs=(argv, system, spline)) as pool:
        pool.map(_pool_task, [np.array([0, 1])] * procs, chunksize=1)  # every process is up and warm
        t0 = time.perf_counter()
        done = sum(pool.imap_unordered(_pool_task, tasks, chunksize=1))
        dt = time.perf_counter() - t0
    return done / dt, done, dt


def host_cpu():
    """(logical cores usable by this process, CPU model name)."""
    import platform

    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return cores, model or platform.processor() or platform.machine()


def cpu_worker(args, argv):
    """Times the FP64 oracle on bounded, seeded samples of centres of the workload: exact radial integrals on one
    host thread and on every host core (a spawned process pool, one thread per process), and the paper's spline
    optimisation (FP64 clamped cubic spline of the same integrals) on every core."""
    import numpy as np

    from oracle import radial as oradial
    from oracle import soap as osoap

    system = make_system(args.config, 0)
    system.hypers = dict(system.hypers, basis=args.basis)
    h = osoap.Hypers(**system.hypers)
    order = np.random.default_rng(123).permutation(system.n_atoms)
    cores, model = host_cpu()
    per_mode = args.cpu_seconds / 3.0
    run = oracle_step_fn(args, system, h)
    run(order[:2])  # first call builds the oracle's per-(a, b) 1F1 switch points
    rate1, n1, dt1, _ = _time_serial(run, order, 2, per_mode)
    modes = [{"radial": "exact 1F1", "cores": 1, "value": rate1, "centres": n1, "seconds": dt1}]
    ratep, npool, dtp = _time_pool(argv, system, None, order, rate1, cores, per_mode) if cores > 1 else (rate1, n1, dt1)
    modes.append({"radial": "exact 1F1", "cores": cores, "value": ratep, "centres": npool, "seconds": dtp})
    if args.basis == "gto":
        spline = oradial.RadialSpline(h.r_cut, h.sigma, h.n_max, h.l_max, accuracy=1e-8, orthonormal=h.orthonormal)
        srun = oracle_step_fn(args, system, h, lambda r, d=False: spline(r, d))
        srun(order[:2])
        rate_s1 = _time_serial(srun, order, 2, 0.25 * per_mode)[0]
        rs, ns, dts = _time_pool(argv, system, spline, order, rate_s1, cores, per_mode) if cores > 1 else \
            _time_serial(srun, order, 2, per_mode)[:3]
        modes.append({"radial": f"FP64 spline ({spline.M} intervals, midpoint error <= 1e-8)", "cores": cores,
                      "value": rs, "centres": ns, "seconds": dts})
    print(json.dumps({"modes": modes, "nproc": cores, "cpu_model": model}))


def gpr_text(args):
    if args.lambda_soap >= 0:
        return f" -> rank-{args.lambda_soap} nu = 2 equivariants instead of p"
    return f" + sparse GPR energy ({args.gpr} sparse points per species, zeta {args.zeta})" if args.gpr else ""


def oracle_gpr_model(args, system, h):
    """The GPR model's sparse points as the oracle computes them (setup, untimed): the drawn atoms' FP64 p."""
    from oracle import soap as osoap
    from synth import gpr_sparse_draws

    idx, x = gpr_sparse_draws(system.species, h.species, args.gpr, seed=31)
    pm = osoap.power_spectrum(osoap.spherical_expansion(system, h, centres=idx), h, "packed").reshape(idx.size, -1)
    return pm, h.species_index(system.species[idx]), x


def oracle_gpr_step(args, system, h, model, centres, radial_fn=None):
    """c, packed p, the GPR energies (and with --gradients dE/dp, forces and virial) of the sampled centres."""
    import numpy as np

    from oracle import gpr as ogpr
    from oracle import soap as osoap

    pm, ms, x = model
    centres = np.asarray(centres)
    cs = h.species_index(system.species[centres])
    p = osoap.power_spectrum(osoap.spherical_expansion(system, h, centres=centres, radial_fn=radial_fn), h,
                             "packed").reshape(centres.size, -1)
    E = ogpr.energies(p, cs, pm, ms, x, args.zeta)
    if args.gradients:
        g = ogpr.grad_p(p, cs, pm, ms, x, args.zeta)
        return E, osoap.energy_gradients(system, h, None, centres=centres, grad_p=g, radial_fn=radial_fn)
    return E


def cpu_baseline(args):
    """The oracle timed on the host cores in a subprocess with no GPU visible (one thread per process)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    argv = ["--config", args.config, "--layout", args.layout, "--cpu-seconds", str(args.cpu_seconds), "--basis",
            args.basis, "--gpr", str(args.gpr), "--zeta", str(args.zeta), "--lambda-soap", str(args.lambda_soap)] + \
        (["--gradients"] if args.gradients else []) + (["--expansion-only"] if args.expansion_only else [])
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-worker"] + argv
    res = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=1200)
    if res.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": None, "kind": "oracle", "error": res.stderr[-300:]}
    d = json.loads(res.stdout.strip().splitlines()[-1])
    modes = d["modes"]
    main = modes[1]  # exact integrals on every host core
    what = (f"neighbours + {'1F1' if args.basis == 'gto' else 'DVR'} coefficients"
            f"{'' if args.expansion_only else ' + ' + args.layout + ' power spectrum'}"
            f"{gpr_text(args)}{' + forces and virial' if args.gradients else ''}, FP64 numpy")
    return {"value": main["value"], "unit": UNIT, "cores": main["cores"], "kind": "oracle",
            "sample": f"{main['centres']} seeded random centres of the {args.config} workload ({what}), exact radial "
                      f"integrals, {main['seconds']:.1f} s on {main['cores']} host processes of one thread each",
            "host": {"nproc": d["nproc"], "cpu_model": d["cpu_model"]},
            "modes": [{k: m[k] for k in ("radial", "cores", "value", "centres", "seconds")} for m in modes]}


def run_reference(args):
    """The reference arm: the FP64 oracle (exact radial integrals) on every host core, a spawned process pool of
    one thread each, each step a bounded seeded sample of the same workload."""
    rank, world, _ = dist_init(args)
    if rank != 0:
        return 0
    import multiprocessing as mp

    import numpy as np

    from oracle import soap as osoap

    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"  # inherited by the spawned processes
    system = make_system(args.config, 0)
    system.hypers = dict(system.hypers, basis=args.basis)
    h = osoap.Hypers(**system.hypers)
    order = np.random.default_rng(7).permutation(system.n_atoms)
    cores, model = host_cpu()
    argv = ["--config", args.config, "--layout", args.layout, "--basis", args.basis, "--gpr", str(args.gpr), "--zeta",
            str(args.zeta), "--lambda-soap", str(args.lambda_soap)] + (["--gradients"] if args.gradients else []) + \
        (["--expansion-only"] if args.expansion_only else [])
    with mp.get_context("spawn").Pool(cores, initializer=_pool_init, initargs=(argv, system, None)) as pool:
        pool.map(_pool_task, [np.array([0, 1])] * cores, chunksize=1)
        t0 = time.perf_counter()
        probe = sum(pool.map(_pool_task, [order[2 + 2 * k:4 + 2 * k] for k in range(cores)], chunksize=1))
        per = (time.perf_counter() - t0) / probe  # wall seconds per centre with every core busy
        budget = args.ref_seconds
        per_step = max(cores, int(budget / max(per, 1e-6) / (args.steps + args.warmup)))
        cursor = 2 + 2 * cores

        def step():
            nonlocal cursor
            idx = np.take(order, np.arange(cursor, cursor + per_step), mode="wrap")
            cursor += per_step
            chunk = max(1, -(-per_step // (4 * cores)))
            return sum(pool.imap_unordered(_pool_task, [idx[k:k + chunk] for k in range(0, per_step, chunk)],
                                           chunksize=1))

        for _ in range(args.warmup):
            step()
        t0 = time.perf_counter()
        done = 0
        for _ in range(args.steps):
            done += step()
        dt = time.perf_counter() - t0
    value = done / dt
    sample = (f"{per_step} seeded random centres per step of the {args.config} workload (neighbours + exact "
              f"{'1F1' if args.basis == 'gto' else 'DVR'} coefficients{'' if args.expansion_only else ' + ' + args.layout + ' power spectrum'}"
              f"{gpr_text(args)}{' + forces and virial' if args.gradients else ''}, "
              f"FP64 numpy), {cores} host processes of one thread each")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.config}: {WORKLOADS[args.config]}", "global_batch": per_step},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "host": {"nproc": cores, "cpu_model": model}},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------------------------------- GPU path
def run_ours(args):
    import torch

    rank, world, local = dist_init(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    import paper_2101_08814_gb300 as rg

    system = make_system(args.config, rank, args.structures)
    system.hypers = dict(system.hypers, basis=args.basis)
    calc = rg.SoapCalculator(**system.hypers, device=dev)
    ds = rg.DeviceSystem.from_numpy(system, device=dev)
    N = ds.n_atoms
    stream = torch.cuda.current_stream(dev)
    Qc = calc.coeffs_per_centre
    Fp = calc.n_features(args.layout)
    if args.gradients and args.select > 0:
        raise SystemExit("--gradients uses the full packed power spectrum; it does not combine with --select")
    if args.gradients and args.layout != "packed":
        raise SystemExit("--gradients uses the linear model over the packed features (--layout packed)")
    coeffs = torch.empty((N, calc.n_species, calc.n_max, (calc.l_max + 1) ** 2), dtype=torch.float32, device=dev)
    sel = None
    if args.select > 0:
        import numpy as np

        Fpk = calc.n_features("packed")
        n_sel = max(1, int(round(args.select * Fpk)))
        sel = torch.tensor(np.sort(np.random.default_rng(11).choice(Fpk, n_sel, replace=False)).astype(np.int32),
                           device=dev)
        Fp = n_sel
    lsoap = None
    if args.lambda_soap >= 0:
        if args.gpr or args.gradients or sel is not None:
            raise SystemExit("--lambda-soap replaces the power spectrum; it does not combine with --gpr/--gradients/--select")
        n_pairs_l, feat_l = calc.lambda_soap_size(args.lambda_soap)
        lsoap = torch.empty((N, n_pairs_l, 2 * args.lambda_soap + 1, calc.n_species * calc.n_max,
                             calc.n_species * calc.n_max), dtype=torch.float32, device=dev)
        Fp = feat_l
    ps = torch.empty((N, Fp if lsoap is None else 1), dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    radial_info = radial_setup(args, calc, system, dev, rg)
    weights = None
    gpr_model, gpr_info = None, None
    if args.gpr:
        if args.layout != "packed" or args.expansion_only:
            raise SystemExit("--gpr takes the packed power spectrum (or a selection of it)")
        gpr_model, gpr_info = gpr_setup(args, calc, system, ds, coeffs, ps, sel, rg)
    if args.gradients and gpr_model is None:
        from synth import linear_weights

        weights = torch.tensor(linear_weights(calc.n_species, calc.n_features("packed"), seed=4), dtype=torch.float32,
                               device=dev)

    def step(events=None):
        # stage boundaries: neighbours | expansion (or fused soap) | power spectrum (separate form) | GPR | gradients
        def mark(k):
            if events is not None:
                events[k].record(stream)

        mark(0)
        pairs = calc.neighbours(ds)
        mark(1)
        if lsoap is not None:
            calc.spherical_expansion(ds, pairs, out=coeffs)
            mark(2)
            calc.lambda_soap(coeffs, args.lambda_soap, out=lsoap)
        elif args.separate or args.expansion_only:
            calc.spherical_expansion(ds, pairs, out=coeffs)
            mark(2)
            if not args.expansion_only:
                calc.power_spectrum(coeffs, precision=args.ps, layout=args.layout, out=ps)
        elif sel is not None:
            calc.soap_selected(ds, pairs, sel, coeffs=coeffs, ps=ps)
            mark(2)
        else:
            calc.soap(ds, pairs, layout=args.layout, precision=args.ps, coeffs=coeffs, ps=ps)
            mark(2)
        mark(3)
        g = None
        if gpr_model is not None:
            _, _, g = gpr_model.predict(ds, ps, grad=args.gradients, atomic=False)
        mark(4)
        if weights is not None:
            calc.linear_energy(ds, ps, weights)
            calc.gradients(ds, pairs, coeffs, weights=weights)
        elif g is not None:
            calc.gradients(ds, pairs, coeffs, grad_ps=g)
        mark(5)
        return pairs

    for _ in range(max(args.warmup, 3)):
        pairs = step()
    torch.cuda.synchronize(dev)
    n_pairs = pairs.n_pairs

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(args.steps)]
    sampler = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    launches0 = rg.launch_count()
    sampler.start()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))  # 256 MB write between steps evicts L2 (129 MB); outside the step's events
        step(evs[k])
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t_wall
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    launches = rg.launch_count() - launches0
    stage = [[e[s].elapsed_time(e[s + 1]) for e in evs] for s in range(5)]
    step_ms = [sum(stage[s][k] for s in range(5)) for k in range(args.steps)]
    ms = sum(step_ms) / len(step_ms)
    ms = max_over_ranks(ms, dev)
    total_env = int(sum_over_ranks(N, dev))
    value = total_env / (ms * 1e-3)

    # roofline of the dominant kernel: algorithmic bytes = inputs read + outputs written (HBM-bound kernels), or
    # algorithmic FP32 flops (the gradient kernel)
    mean = [sum(x) / len(x) for x in stage]
    pair_in = 24 * n_pairs + 8 * (N + 1)                      # r_ji float4 + j + species(j); CSR offsets
    c_bytes = 4 * Qc * N
    p_bytes = 4 * Fp * N
    fused = not (args.separate or args.expansion_only or lsoap is not None)
    peak, peak_kind = load_peaks()
    peak_src = f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback 6.8 TB/s"
    cand = {"rascal_neighbours": (None, mean[0])}
    if fused:
        cand["k_expansion<fused power spectrum> (rascal_soap)"] = (pair_in + c_bytes + p_bytes, mean[1])
    else:
        cand["k_expansion (rascal_spherical_expansion)"] = (pair_in + c_bytes, mean[1])
        if lsoap is not None:
            cand["k_lambda_soap (rascal_lambda_soap)"] = (c_bytes + 4 * lsoap.numel(), mean[2])
        elif not args.expansion_only:
            cand["power spectrum (rascal_power_spectrum)"] = (c_bytes + p_bytes, mean[2])
    if gpr_model is not None:
        cand["rascal_gpr_predict (k_gpr_kernel" + (" + k_gpr_grad)" if args.gradients else ")")] = (None, mean[3])
    if args.gradients:
        cand["k_gradients (" + ("rascal_gradients on dE/dp)" if gpr_model is not None else
                                "rascal_linear_energy + rascal_gradients)")] = (None, mean[4])
    kernel = max(cand, key=lambda k: cand[k][1])
    alg, t_ms = cand[kernel]
    if kernel.startswith("rascal_gpr_predict"):
        flops = gpr_info["flops_energy"] * (2 if args.gradients else 1)
        bf16, tf32_kind = load_tensor_peak()
        tf32_peak = bf16 * 1.1 / 2.25
        achieved = flops / (t_ms * 1e-3) / 1e12
        roofline = {"bound": "tensor", "kernel": kernel, "achieved": achieved, "peak": tf32_peak, "unit": "TFLOP/s",
                    "frac": achieved / tf32_peak, "traffic": None, "algorithmic_flops_per_launch": flops,
                    "peak_source": f"TF32 = {tf32_kind} bf16 peak x 1.1/2.25 (nominal dense TF32/BF16 ratio); the "
                                   "timed region is the whole call (species sort, GEMMs, finish)"}
    elif kernel.startswith("k_gradients"):
        # per pair: s += chat dR Y and w += chat R grad Y over the centre's species block, 2 + 3 FMA per (n, lm);
        # per centre: the adjoint chat_l = k_l (W + W^T) C_l, Q x Q times Q x (2l+1)
        n_lm = (calc.l_max + 1) ** 2
        Q = calc.n_species * calc.n_max
        flops = 10.0 * calc.n_max * n_lm * n_pairs + 2.0 * Q * Q * n_lm * N
        sm_max = (clocks or {}).get("sm_max_mhz") or 2070.0
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        alu_peak = n_sm * 128 * 2 * sm_max * 1e6 / 1e12  # FP32 FMA lanes x 2 flop x max SM clock, TFLOP/s
        achieved = flops / (t_ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                    "frac": achieved / alu_peak, "traffic": None, "algorithmic_flops_per_launch": flops,
                    "peak_source": f"FP32 FMA peak from unit counts: {n_sm} SMs (device properties) x 128 lanes x "
                                   "2 flop x max SM clock"}
    else:
        achieved = (alg / (t_ms * 1e-3) / 1e9) if alg else None
        traffic_known = (kernel.startswith("k_expansion<fused") and args.config == "batch" and args.ps == "fp32"
                         and args.layout == "packed" and args.radial == "spline" and sel is None)
        roofline = {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": (achieved / peak) if achieved else None,
                    "traffic": FUSED_FP32_TRAFFIC_PER_ENV * N if traffic_known and FUSED_FP32_TRAFFIC_PER_ENV else None,
                    "algorithmic_bytes_per_launch": alg, "peak_source": peak_src}
    if radial_info.get("check_error"):
        radial_info["c_err_vs_exact_fp64"] = coefficient_error(calc, ds, coeffs, rg, args)
        del radial_info["check_error"]

    e2e = None
    if lsoap is not None:
        # the equivariants are GBs per step: reading them back every step would time the PCIe/C2C link alone
        args.no_e2e = True
    if not args.no_e2e and world >= 1:
        e2e = measure_e2e(args, calc, system, dev, stream, ps, coeffs, rg, weights=weights, sel=sel, gpr=gpr_model)
        e2e["ms"] = max_over_ranks(e2e["ms"], dev)
        e2e = {"value": total_env / (e2e["ms"] * 1e-3), "unit": UNIT, "h2d_bytes_per_step": e2e["h2d"],
               "d2h_bytes_per_step": e2e["d2h"], "ms_per_step": e2e["ms"]}

    if rank == 0:
        cpu = None if args.no_cpu_baseline or world > 1 else cpu_baseline(args)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"{args.config}: {WORKLOADS[args.config]}", "global_batch": total_env,
                       "env_per_gpu": N, "pairs_per_gpu": n_pairs,
                       **({"lambda_soap": {"lambda": args.lambda_soap, "features": Fp}} if lsoap is not None else {}),
                       "power_spectrum": None if (args.expansion_only or lsoap is not None) else {"layout": args.layout,
                                                                                                   "precision": args.ps,
                                                                          "fused": fused, "features": Fp,
                                                                          "selected": sel is not None},
                       "gradients": bool(args.gradients), "radial_basis": args.basis, **radial_info,
                       **({"gpr": gpr_info["config"]} if gpr_info else {}),
                       "parallelism": f"dp{world} (independent batches per GPU)",
                       "l2": "256 MB buffer written before every timed step (L2 is 129 MB), outside the step events",
                       "stage_ms": {"neighbours": mean[0], ("expansion" if not fused else "soap"): mean[1],
                                    **({"power_spectrum": mean[2]} if args.separate else {}),
                                    **({"lambda_soap": mean[2]} if lsoap is not None else {}),
                                    **({"gpr": mean[3]} if gpr_model is not None else {}),
                                    **({"gradients": mean[4]} if args.gradients else {})},
                       "wall_ms_per_step_incl_flush": 1e3 * wall / args.steps},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
        }
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def radial_setup(args, calc, system, dev, rg):
    """Selects the radial source. The MLP surrogate is trained on the GPU first (setup, outside the timed steps)."""
    import torch

    info = {"radial": args.radial}
    if args.radial == "exact":
        calc.set_radial("exact")
    elif args.radial == "mlp":
        from synth import mlp_initial_params, mlp_training_draws

        F = calc.n_max * (calc.l_max + 1)
        r_cut = float(system.hypers["r_cut"])
        batch = 4096
        r, order = mlp_training_draws(1 << 20, r_cut, batch, args.mlp_steps, seed=22)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        tgt, scale = calc.mlp_targets(torch.tensor(r))
        calc.mlp_set_params(mlp_initial_params(calc.MLP_HIDDEN, F, seed=23), scale)
        t = torch.tensor(r / r_cut, dtype=torch.float32, device=dev)
        loss = calc.mlp_train(t, tgt, torch.tensor(order, device=dev), batch=batch, steps=args.mlp_steps, lr_max=1e-2,
                              lr_min=1e-5, total_steps=args.mlp_steps)
        torch.cuda.synchronize(dev)
        info.update({"mlp_training": f"{args.mlp_steps} Adam steps (batch {batch}, cosine lr 1e-2 -> 1e-5) on 2^20 "
                                     f"FP64-exact samples, r uniform in [0, {r_cut}] A",
                     "mlp_setup_s": time.perf_counter() - t0, "mlp_final_loss": float(loss[-1].item())})
        calc.set_radial("mlp")
        info["check_error"] = True
    return info


def coefficient_error(calc, ds, coeffs, rg, args):
    """Block max-relative errors of c (per centre and species block, max |dc| / max |c_ref|) of the timed radial
    source and of the spline, both against the per-pair FP64 exact-1F1 path on the same GPU."""
    def err(c, ref):
        d = (c - ref).abs().flatten(2).amax(dim=2)
        m = ref.abs().flatten(2).amax(dim=2)
        ok = m > 0
        return float((d[ok] / m[ok]).max().item())

    pairs = calc.neighbours(ds)
    calc.set_radial("exact")
    ref = calc.spherical_expansion(ds, pairs)
    calc.set_radial("spline")
    spline = calc.spherical_expansion(ds, pairs)
    calc.set_radial(args.radial)
    mine = calc.spherical_expansion(ds, pairs)
    return {args.radial: err(mine, ref), "spline": err(spline, ref)}


def measure_e2e(args, calc, system, dev, stream, ps, coeffs, rg, steps=None, weights=None, sel=None, gpr=None):
    """Same step through the public API with host buffers: pinned H2D of the inputs, D2H of the power spectrum.

    Steps are pipelined the way a streaming user would run them: the power spectrum of step k leaves on a copy
    stream while step k + 1 computes into the other of two output buffers; each buffer is reused only after its
    copy has finished. Every step's inputs go host -> device and every step's p goes device -> host inside the
    timed region.
    """
    import torch

    steps = steps or max(3, min(args.steps, 20))
    host = {
        "positions": torch.as_tensor(system.positions, dtype=torch.float64).pin_memory(),
        "species": torch.as_tensor(system.species, dtype=torch.int32).pin_memory(),
        "cells": torch.as_tensor(system.cells, dtype=torch.float64).pin_memory(),
        "pbc": torch.as_tensor(system.pbc, dtype=torch.int32).pin_memory(),
        "struct_offsets": torch.as_tensor(system.struct_offsets, dtype=torch.int32).pin_memory(),
    }
    dev_t = {k: torch.empty_like(v, device=dev) for k, v in host.items()}
    result = coeffs if args.expansion_only else ps  # the step's result read back by the host
    if gpr is not None:  # the model's structure energies are the result; p stays on the device
        result = torch.empty(system.n_structures, dtype=torch.float64, device=dev)
    ps_buf = [result, torch.empty_like(result)]
    out_host = [torch.empty(result.shape, dtype=result.dtype).pin_memory() for _ in range(2)]
    forces_host = torch.empty((system.n_atoms, 3), dtype=torch.float64).pin_memory()
    ds = rg.DeviceSystem(dev_t["positions"], dev_t["species"], dev_t["cells"], dev_t["pbc"], dev_t["struct_offsets"])
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    d2h = out_host[0].numel() * out_host[0].element_size() + \
        (forces_host.numel() * 8 if (weights is not None or (gpr is not None and args.gradients)) else 0)
    copy_stream = torch.cuda.Stream(dev)
    copied = [None, None]

    def one(k):
        b = k & 1
        cur = torch.cuda.current_stream(dev)
        if copied[b] is not None:
            cur.wait_event(copied[b])
        for key in host:
            dev_t[key].copy_(host[key], non_blocking=True)
        pairs = calc.neighbours(ds)
        forces = None
        if gpr is not None:  # p stays on the device; the result buffers hold the structure energies
            if args.separate:
                calc.spherical_expansion(ds, pairs, out=coeffs)
                calc.power_spectrum(coeffs, precision=args.ps, layout=args.layout, out=ps)
            elif sel is not None:
                calc.soap_selected(ds, pairs, sel, coeffs=coeffs, ps=ps)
            else:
                calc.soap(ds, pairs, layout=args.layout, precision=args.ps, coeffs=coeffs, ps=ps)
        elif args.expansion_only:
            calc.spherical_expansion(ds, pairs, out=ps_buf[b])
        elif args.separate:
            calc.spherical_expansion(ds, pairs, out=coeffs)
            calc.power_spectrum(coeffs, precision=args.ps, layout=args.layout, out=ps_buf[b])
        elif sel is not None:
            calc.soap_selected(ds, pairs, sel, coeffs=coeffs, ps=ps_buf[b])
        else:
            calc.soap(ds, pairs, layout=args.layout, precision=args.ps, coeffs=coeffs, ps=ps_buf[b])
        if gpr is not None:
            e, _, g = gpr.predict(ds, ps, grad=args.gradients, atomic=False)
            ps_buf[b].copy_(e)
            if g is not None:
                forces, _ = calc.gradients(ds, pairs, coeffs, grad_ps=g)
        elif weights is not None:
            calc.linear_energy(ds, ps_buf[b], weights)
            forces, _ = calc.gradients(ds, pairs, coeffs, weights=weights)
        ready = torch.cuda.Event()
        ready.record(cur)
        copy_stream.wait_event(ready)
        with torch.cuda.stream(copy_stream):
            out_host[b].copy_(ps_buf[b], non_blocking=True)
            if forces is not None:
                forces_host.copy_(forces, non_blocking=True)
        copied[b] = torch.cuda.Event()
        copied[b].record(copy_stream)

    for k in range(2):
        one(k)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for k in range(steps):
        one(k)
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    return {"ms": 1e3 * dt / steps, "h2d": h2d, "d2h": d2h}


def main(argv=None):
    args = parse_args(argv)
    if args.cpu_worker:
        cpu_worker(args, [a for a in (sys.argv[1:] if argv is None else argv) if a != "--cpu-worker"])
        return 0
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
