"""Benchmark: GSE-TDVP1 time steps per second on one GB300 (and the oracle on CPU).

One timed step = one full GSE-TDVP1 time step (Sec. I.C: Krylov vectors of
Eq. 10, basis extension of Eqs. 3-7, symmetric TDVP1 sweep) on the 4 x 16
Heisenberg cylinder (snake path, MPO bond dimension up to 14), starting from a
synthetic state that is already resident in HBM.  The state is reset to the
same synthetic input before every timed step, so every step does identical
work.  H_eff applies run on the tcgen05 split-TF32 path; Lanczos, gauge moves
and the density-matrix steps run in FP64.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--chi0 C] [--chi-max X]
    python bench.py --impl reference ...      (the CPU oracle on the host cores)

Under torchrun each rank evolves its own independent copy (replicas only:
a single chain's sweep does not shard); rank 0 prints one JSON line.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GSE-TDVP1 sweeps/s and H_eff TFLOP/s at chi=1024, precision vs FP64 GPU, at <=1e-7 energy err"
UNIT = "sweeps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--chi0", type=int, default=32, help="bond dimension of the synthetic start state")
    ap.add_argument("--chi-max", type=int, default=64)
    ap.add_argument("--k", type=int, default=3)
    ap.add_argument("--dt", type=float, default=0.1)
    ap.add_argument("--heff-chi", type=int, default=1024, help="bond dimension of the H_eff roofline probe")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--heff-probe", action="store_true",
                    help="only time the tensor-core H_eff apply at --heff-chi (the profiling target)")
    return ap.parse_args()


def workload(args):
    from paper_2005_06104_gb300 import workloads as wl
    lat = wl.cylinder_snake(16, 4)
    W = wl.heisenberg_mpo(lat)
    psi = wl.random_mps(lat.n, args.chi0, seed=2024)
    nrm = np.sqrt(abs(_overlap(psi, psi)))
    psi[0] = psi[0] / nrm
    cfg = {"workload": f"heisenberg_cylinder4x16_snake_w14_chi0_{args.chi0}_chimax_{args.chi_max}_k{args.k}",
           "lattice": "4x16 cylinder, snake path, J=1", "n_sites": lat.n, "mpo_bond_dim_max": 14,
           "chi0": args.chi0, "chi_max": args.chi_max, "krylov_order_k": args.k, "dt": args.dt,
           "tau": args.dt, "eps_k": 1e-8, "eps_m": 1e-8, "eps": 0.0, "time": "real",
           "heff_precision": "tf32x3", "start_state": "random dense MPS (seed 2024), normalised",
           "l2": "working set > L2 per step (environments + Krylov vectors); no flush"}
    return lat, W, psi, cfg


def _overlap(a, b):
    E = np.ones((1, 1), dtype=np.complex128)
    for x, y in zip(a, b):
        T = np.tensordot(E, y, axes=([1], [0]))
        E = np.tensordot(x.conj(), T, axes=([0, 1], [0, 1]))
    return complex(E[0, 0])


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.path = tempfile.mktemp(suffix=".csv")
        self.idx = gpu_index
        self.proc = None

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(args, W, psi, budget_s=20.0):
    """The oracle (as it stands) on the host cores: one H_eff-dominated sample of the
    same step, scaled to sweeps/s by the GPU step's own count of H_eff applies."""
    import oracle as O
    t0 = time.perf_counter()
    p = dict(tau=args.dt, k=args.k, eps_k=1e-8, eps_m=1e-8, chi_max=args.chi_max, dt=args.dt,
             kind="real", eps=0.0)
    # time a whole oracle step when it fits the budget, else the TDVP1 part of one site
    stats = {}
    psi_c = O.left_canonicalize(psi)
    t = time.perf_counter()
    out = O.gse_tdvp1_step(psi_c, W, p, stats)
    dt_step = time.perf_counter() - t
    sample = f"one full GSE-TDVP1 step of the same workload ({len(stats.get('lanczos_iters', []))} local exponentials)"
    if time.perf_counter() - t0 > budget_s * 3:
        sample += " (exceeded the sampling budget)"
    del out
    return {"value": 1.0 / dt_step, "unit": UNIT, "cores": _blas_threads(), "kind": "oracle", "sample": sample,
            "seconds": dt_step}


def _blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads") for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(n[0])
    except Exception:
        pass
    return os.cpu_count()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    lat, W, psi, cfg = workload(args)
    import oracle as O
    p = dict(tau=args.dt, k=args.k, eps_k=1e-8, eps_m=1e-8, chi_max=args.chi_max, dt=args.dt,
             kind="real", eps=0.0)
    psi_c = O.left_canonicalize(psi)
    for _ in range(args.warmup):
        O.gse_tdvp1_step(psi_c, W, p)
    ts = []
    for _ in range(args.steps):
        t = time.perf_counter()
        O.gse_tdvp1_step(psi_c, W, p)
        ts.append(time.perf_counter() - t)
    total = sum(ts)
    v = args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": _blas_threads(), "kind": "oracle",
                             "sample": "full GSE-TDVP1 steps of the same workload (NumPy complex128)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def heff_roofline(g, torch, chi, W):
    """Timed H_eff applies at bond dimension chi on the 14-wide MPO site (tensor-core path),
    CUDA events on the launching stream."""
    gen = torch.Generator(device="cuda").manual_seed(7)

    def rnd(*s):
        return torch.complex(torch.randn(*s, generator=gen, device="cuda", dtype=torch.float64),
                             torch.randn(*s, generator=gen, device="cuda", dtype=torch.float64))
    L, R, x = rnd(chi, W.shape[0], chi), rnd(chi, W.shape[3], chi), rnd(chi, 2, chi)
    y = torch.empty_like(x)
    nnz = int(np.count_nonzero(W))
    flops = 8.0 * (chi * 2 * chi * (chi * W.shape[0] + chi * W.shape[3]) + chi * chi * nnz)
    st = torch.cuda.current_stream()
    for _ in range(3):
        g.heff_contract(L, W, R, x, y, g.PREC_TF32X3, stream=st.cuda_stream)
    reps = 10
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(st)
    for _ in range(reps):
        g.heff_contract(L, W, R, x, y, g.PREC_TF32X3, stream=st.cuda_stream)
    b.record(st)
    b.synchronize()
    ms = a.elapsed_time(b) / reps
    # bytes that must cross HBM at least once: L, R, x (complex128 in) and y out
    return flops, ms


def run_gpu(args):
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2005_06104_gb300 import gse_tdvp as g
    lat, W, psi, cfg = workload(args)
    opts = dict(tau=args.dt, eps_k=1e-8, eps_m=1e-8, eps=0.0, chi_max=args.chi_max, precision=g.PREC_TF32X3)
    stream = torch.cuda.current_stream().cuda_stream
    st = g.GseTdvp(psi, W, stream=stream, **opts)
    init = st.get_mps()  # the canonical synthetic input, re-uploaded before each step

    def step():
        st.expand_basis(args.k)
        st.sweep(args.dt, g.REAL)

    def reset():
        nonlocal st
        st.close()
        st = g.GseTdvp(init, W, stream=stream, **opts)

    for _ in range(args.warmup):
        step()
        reset()
    clocks = Clocks(local)
    e0 = None
    ts = []
    heff_ms = heff_flops = 0.0
    heff_n = 0
    nfo = {}
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    phases = {}
    for _ in range(args.steps):
        st.profile(True)
        st.trace(True)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        step()
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b))
        pr = st.profile_read()
        for kk, vv in st.trace_read().items():
            phases[kk] = phases.get(kk, 0.0) + vv / args.steps
        heff_ms += pr["ms"]
        heff_flops += pr["flops"]
        heff_n += pr["applies"]
        nfo = st.trunc_stats()
        nfo["bond_dim_max"] = max(st.bond_dims())
        reset()
    torch.cuda.synchronize()
    ck = clocks.stop()
    t_rank = sum(ts) / 1e3
    if world > 1:
        tt = torch.tensor([t_rank], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_rank = tt.item()
    value = world * args.steps / t_rank
    # precision vs FP64: one step in each form from the same input
    e_tc = e_64 = None
    if rank == 0:
        a = g.GseTdvp(init, W, stream=stream, **dict(opts, precision=g.PREC_FP64))
        a.expand_basis(args.k)
        a.sweep(args.dt, g.REAL)
        e_64 = a.energy()
        a.close()
        b_ = g.GseTdvp(init, W, stream=stream, **opts)
        b_.expand_basis(args.k)
        b_.sweep(args.dt, g.REAL)
        e_tc, n_tc = b_.energy(), b_.norm()
        b_.close()
    # e2e: host state in (pinned copy), one step through the public API, full state out
    e2e_ts = []
    h2d = sum(a.nbytes for a in init) + sum(w.nbytes for w in W)
    d2h = 0
    for _ in range(max(1, min(args.steps, 2))):
        torch.cuda.synchronize()
        t = time.perf_counter()
        s2 = g.GseTdvp(init, W, stream=stream, **opts)
        s2.expand_basis(args.k)
        s2.sweep(args.dt, g.REAL)
        out = s2.get_mps()
        s2.close()
        e2e_ts.append(time.perf_counter() - t)
        d2h = sum(a.nbytes for a in out)
    # H_eff roofline probe at chi = heff_chi
    Wmax = max(W, key=lambda w: w.shape[0] * w.shape[3])
    pflops, pms = heff_roofline(g, torch, args.heff_chi, Wmax)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else None
    bf16 = peaks["bf16_tflops"] if peaks else 1900.0
    tf32_peak = bf16 * (1.1 / 2.25)  # measured bf16 x nominal tf32/bf16 ratio
    if rank != 0:
        st.close()
        return
    cpu = None
    if not args.no_cpu_baseline:
        try:
            cpu = cpu_baseline(args, W, init)
        except Exception as ex:  # reported, never silently replaced
            cpu = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": f"failed: {ex}"}
    achieved_step = heff_flops / (heff_ms / 1e3) / 1e12 if heff_ms > 0 else None
    achieved = pflops / (pms / 1e3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sum(ts) / len(ts), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c128 state / tf32x3 H_eff", "data": "synthetic",
        "config": dict(cfg, parallelism=f"replicas{world}"),
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": tf32_peak, "unit": "TFLOP/s",
                     "frac": achieved / tf32_peak, "traffic": None,
                     "kernel": f"H_eff apply (tcgen05 kind::tf32, 3 split products) at chi={args.heff_chi}, w=14",
                     "peak_source": "MEASURED_PEAKS bf16_tflops x 1.1/2.25 (nominal tf32/bf16)",
                     "ms_per_apply": pms, "algorithmic_flops_per_apply": pflops},
        "heff_in_step": {"applies": heff_n, "ms": heff_ms, "tflops_algorithmic": achieved_step,
                         "share_of_step": heff_ms / sum(ts) if ts else None},
        "precision_vs_fp64": {"energy_tf32x3": e_tc, "energy_fp64": e_64,
                              "rel_energy_err": abs(e_tc - e_64) / abs(e_64) if e_64 else None,
                              "norm_drift": abs(n_tc - 1.0)},
        "step_stats": nfo,
        "phases_ms_per_step": phases,
        "cpu_baseline": cpu,
        "e2e": {"value": len(e2e_ts) / sum(e2e_ts), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "what": "tdvp_create from host MPS + expand + sweep + tdvp_get_mps + destroy"},
        "gpu_launches": None,
        "clocks": ck,
    }
    print(json.dumps(line), flush=True)
    st.close()
    if world > 1:
        dist.destroy_process_group()


def run_heff_probe(args):
    import torch
    from paper_2005_06104_gb300 import gse_tdvp as g
    from paper_2005_06104_gb300 import workloads as wl
    W = max(wl.heisenberg_mpo(wl.cylinder_snake(16, 4)), key=lambda w: w.shape[0] * w.shape[3])
    flops, ms = heff_roofline(g, torch, args.heff_chi, W)
    print(json.dumps({"heff_chi": args.heff_chi, "w": int(W.shape[0]), "ms_per_apply": ms,
                      "algorithmic_tflops": flops / ms / 1e9}), flush=True)


def main():
    args = parse()
    if args.heff_probe:
        run_heff_probe(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
