"""Benchmark: GSE-TDVP1 time steps per second on one GB300 (and the oracle on CPU).

One timed step = one full GSE-TDVP1 time step (Sec. I.C: Krylov vectors of
Eq. 10, basis extension of Eqs. 3-7, symmetric TDVP1 sweep) on the 4 x 16
Heisenberg cylinder (snake path, MPO bond dimension up to 14) along the real-time
trajectory from the Neel state with one flipped spin; the state is resident in
HBM.  Untimed preparation and warm-up steps grow the bond dimension to chi_max
(1024 by default) first.  The precision form (BF16X10 by default) runs H_eff,
K_eff, the environment updates and the Krylov GEMMs on the tcgen05 tensor cores;
Lanczos, SVDs and observables are FP64.  The FP64 comparison and the TDVP2
comparison run on a second trajectory capped at --compare-chi (256).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--chi-max X] [--prep-steps P]
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

T_START = time.time()
METRIC = "GSE-TDVP1 sweeps/s and H_eff TFLOP/s at chi=1024, precision vs FP64 GPU, at <=1e-7 energy err"
UNIT = "sweeps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--chi-max", type=int, default=1024)
    ap.add_argument("--compare-chi", type=int, default=256,
                    help="bond-dimension cap of the trajectory that carries the FP64 and TDVP2 comparisons")
    ap.add_argument("--prep-steps", type=int, default=9,
                    help="untimed GSE-TDVP1 steps that grow the bond dimension before warm-up")
    ap.add_argument("--compare-prep", type=int, default=10,
                    help="steps of the comparison trajectory before its FP64 / precision-form / TDVP2 steps")
    ap.add_argument("--time-budget", type=float, default=1650.0,
                    help="wall-clock seconds the whole run may take: the timed loop stops early (and says so) "
                         "when the steps left and the e2e step would not fit")
    ap.add_argument("--k", type=int, default=3)
    ap.add_argument("--krylov", default="dm", choices=["dm", "zipup"],
                    help="Krylov vectors by the density-matrix algorithm (default) or by zip-up")
    ap.add_argument("--dt", type=float, default=0.1)
    ap.add_argument("--heff-chi", type=int, default=1024, help="bond dimension of the H_eff roofline probe")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tdvp2", action="store_true", help="skip the TDVP2 step of the comparison")
    ap.add_argument("--config2", action="store_true",
                    help="imaginary time on the rung-decoupled 2 x 20 ladder, 50 steps, FP64 / TF32X3 / BF16X10")
    ap.add_argument("--config3", action="store_true",
                    help="real time on the 2 x 50 ladder, chi <= 512, 40 BF16X10 steps with per-step FP64 checks")
    ap.add_argument("--peaks", action="store_true",
                    help="measure the FP64 / FP32 / TF32 / complex128 library matmul rates (roofline denominators)")
    ap.add_argument("--oat", action="store_true",
                    help="one-axis twisting at N = 100 (Fig. 4 setting) against the exact Dicke-subspace solution")
    ap.add_argument("--oat-chi", type=int, default=256, help="bond-dimension cap of the --oat runs")
    ap.add_argument("--fig3", action="store_true",
                    help="imaginary time on the rung-decoupled ladder (Fig. 3): GSE-TDVP1 at d tau 0.1 and 0.4, TDVP2")
    ap.add_argument("--fig3-leg", type=int, default=20, help="leg length of the --fig3 ladder")
    ap.add_argument("--fig3-tau", type=float, default=4.0, help="imaginary time of the --fig3 runs")
    ap.add_argument("--svd-probe", action="store_true",
                    help="time only the blocked Jacobi SVDs of tdvp_create on a dense random MPS (bond --heff-chi)")
    ap.add_argument("--u1", action="store_true",
                    help="with --heff-probe: operands with the zero pattern of U(1) charges")
    ap.add_argument("--heff-probe", action="store_true",
                    help="only time the tensor-core H_eff apply at --heff-chi (the profiling target)")
    ap.add_argument("--precision", default="bf16x10", choices=sorted(PRECISIONS),
                    help="arithmetic of the dense contractions (Lanczos, SVDs, observables stay FP64)")
    ap.add_argument("--krylov-precision", default="bf16x6", choices=sorted(PRECISIONS) + ["same"],
                    help="arithmetic of the Krylov vectors' contractions in the precision form ('same': "
                         "--precision); FP64 handles always run FP64")
    ap.add_argument("--batch-chains", type=int, default=0,
                    help="time the batch workload instead: this many random-field chains (lengths 20-60, "
                         "chi_max 32-128, dt 0.05, k 2) stepped together, against the same chains one at a time")
    ap.add_argument("--batch-threads", type=int, default=0, help="host workers of the batch (0: all cores)")
    ap.add_argument("--step-only", action="store_true",
                    help="stop after the timed steps (no FP64 comparison, e2e, probe or CPU baseline): "
                         "the short command a launch-list profile runs")
    return ap.parse_args()


PRECISIONS = {"fp64": "PREC_FP64", "tf32x3": "PREC_TF32X3", "tf32x3_env": "PREC_TF32X3_ENV",
              "bf16x10": "PREC_BF16X10", "bf16x6": "PREC_BF16X6"}
PRECISION_TEXT = {
    "fp64": "FP64 on CUDA cores throughout",
    "tf32x3": "tcgen05 split TF32 x3 (H_eff, K_eff, Krylov GEMMs); FP64 environments, Lanczos, SVD",
    "tf32x3_env": "tcgen05 split TF32 x3 (H_eff, K_eff, environments, Krylov GEMMs); FP64 Lanczos, SVD",
    "bf16x10": "tcgen05 BF16 exact slices x10 (H_eff, K_eff, environments, Krylov GEMMs); FP64 Lanczos, QR, SVD, "
               "eigendecompositions",
    "bf16x6": "tcgen05 BF16 exact slices x6 (H_eff, K_eff, environments, Krylov GEMMs); FP64 Lanczos, QR, SVD; "
              "Krylov density matrices: FP64 pivoted Cholesky, FP32 Jacobi rotations",
}


def prec_code(g, name):
    return getattr(g, PRECISIONS[name])


def workload(args):
    """The 4 x 16 Heisenberg cylinder (snake path) from Neel with the spin at (8, 0) flipped,
    real time dt = 0.1, k = 3: the trajectory is advanced untimed (--prep-steps) until its
    bond dimensions approach chi_max, then the timed steps continue the same trajectory."""
    from paper_2005_06104_gb300 import workloads as wl
    lat = wl.cylinder_snake(16, 4)
    W = wl.heisenberg_mpo(lat)
    psi = wl.neel_state(lat, flip=(8, 0))
    cfg = {"workload": f"heisenberg_cylinder4x16_snake_neel_flip_chimax{args.chi_max}_k{args.k}_dt{args.dt}",
           "lattice": "4x16 cylinder (periodic in y), snake path, J=1", "n_sites": lat.n,
           "mpo_bond_dim_max": int(max(wl.mpo_bond_dims(W))), "chi_max": args.chi_max,
           "krylov_order_k": args.k, "dt": args.dt, "tau": args.dt, "eps_k": 1e-8, "eps_m": 1e-8, "eps": 0.0,
           "time": "real", "precision_form": PRECISION_TEXT[args.precision],
           "krylov_precision": args.precision if args.krylov_precision == "same" else args.krylov_precision,
           "start_state": "Neel with the spin at (8,0) flipped", "prep_steps": args.prep_steps,
           "compare_chi": args.compare_chi, "krylov_method": "density_matrix" if args.krylov == "dm" else "zipup",
           "l2": "working set of a step (environments, Krylov vectors, density environments) > L2; no flush"}
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


def _lanczos_iters_oracle(args, W, chi=32):
    """Mean Krylov dimension per local exponential of the oracle's TDVP1 sweep on the same
    lattice and time step at a small bond dimension (the count depends on dt and the
    spectral width of H, not on chi)."""
    import oracle as O
    from paper_2005_06104_gb300 import workloads as wl
    psi = O.right_canonicalize(wl.random_mps(len(W), chi, seed=11))
    psi[0] = psi[0] / np.linalg.norm(psi[0])
    st = {}
    O.tdvp1_sweep(psi, W, args.dt, "real", stats=st)
    return float(np.mean(st["lanczos_iters"]))


def cpu_baseline(args, W, iters=None):
    """The oracle (as it stands) on the host cores, on a bounded sample of one sweep at the
    bench's bond dimension: its primitives timed once each at the centre site's shapes (bond
    dimension min(chi_max, 2^(N/2)), MPO width of the centre): one H_eff apply, one K_eff
    apply, one block QR (the real-time gauge move) and one environment update.  The sweep is
    extrapolated from that sample: a site update = iters H_eff applies + iters K_eff applies +
    QR + update, scaled to the 2N site updates by each site's m_l m_r (m_l + m_r) share.
    iters: Krylov dimension per local exponential, from _lanczos_iters_oracle.  Steps 1-2
    (Krylov vectors, extension) are left out, which favours the CPU."""
    import oracle as O
    from paper_2005_06104_gb300 import workloads as wl
    n = len(W)
    c = n // 2
    dims = wl.full_bond_dims(n, args.chi_max)
    m, wc, wr = dims[c], W[c].shape[0], W[c].shape[3]
    rng = np.random.default_rng(11)

    def rnd(*shape):
        return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(np.prod(shape))
    A, L, R = rnd(m, 2, m), rnd(m, wc, m), rnd(m, wr, m)
    C, Lb = rnd(m, m), rnd(m, wr, m)
    if iters is None:
        iters = _lanczos_iters_oracle(args, W)

    def timed(f):
        t = time.perf_counter()
        f()
        return time.perf_counter() - t
    t0 = time.perf_counter()
    t_heff = timed(lambda: O.heff_apply(L, W[c], R, A))
    t_keff = timed(lambda: O.keff_apply(Lb, R, C))
    t_qr = timed(lambda: O.qr_blocks(A.reshape(2 * m, m)))
    t_env = timed(lambda: O.env_left_step(L, A, W[c]))
    sample_s = time.perf_counter() - t0
    t_site = iters * (t_heff + t_keff) + t_qr + t_env
    cost = [dims[i] * dims[i + 1] * (dims[i] + dims[i + 1]) for i in range(n)]
    t_sweep = 2.0 * t_site * sum(cost) / cost[c]
    return {"value": 1.0 / t_sweep, "unit": UNIT, "cores": _blas_threads(),
            "kind": "oracle: timed sample at chi_max, extrapolated to one sweep (Krylov and extension excluded)",
            "sample": f"oracle primitives at the centre site (chi={m}, w={wc}) timed once each: H_eff apply "
                      f"{t_heff:.2f} s, K_eff apply {t_keff:.2f} s, block QR {t_qr:.2f} s, environment update "
                      f"{t_env:.2f} s; a site update = {iters:.1f} Krylov iterations (the oracle's own mean on "
                      f"this lattice and dt at chi=32) of H_eff and of K_eff + QR + update; scaled to one sweep "
                      f"by m_l m_r (m_l+m_r); Krylov and extension steps excluded (favours the CPU)",
            "sample_s": sample_s, "seconds_per_site_update": t_site, "extrapolated_s_per_sweep": t_sweep}


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
    """The oracle on the host cores (rank 0 only; other ranks exit without work).  Each step
    is one bounded sample of the chi_max workload (cpu_baseline: the oracle's primitives at the
    centre site, timed); ms_per_step is the measured wall time of a sample, and value is the
    sweep rate extrapolated from the samples (labelled as such in cpu_baseline.kind)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    lat, W, psi, cfg = workload(args)
    iters = _lanczos_iters_oracle(args, W)
    for _ in range(args.warmup):
        cpu_baseline(args, W, iters)
    samples = [cpu_baseline(args, W, iters) for _ in range(args.steps)]
    t_sweep = [x["extrapolated_s_per_sweep"] for x in samples]
    v = args.steps / sum(t_sweep)
    cb = dict(samples[-1])
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(x["sample_s"] for x in samples) / args.steps,
            "ms_per_step_is": "measured wall time of one timed sample (the value is extrapolated from it)",
            "extrapolated_ms_per_sweep": 1e3 * sum(t_sweep) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": cfg, "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def heff_roofline(g, torch, chi, W, prec):
    """Timed H_eff applies at bond dimension chi on the 14-wide MPO site, CUDA events on the
    launching stream.  Returns (algorithmic flops, ms per apply with the environment operands
    cached as inside a Lanczos run, ms per apply rebuilding them every call)."""
    gen = torch.Generator(device="cuda").manual_seed(7)

    def rnd(*s):
        return torch.complex(torch.randn(*s, generator=gen, device="cuda", dtype=torch.float64),
                             torch.randn(*s, generator=gen, device="cuda", dtype=torch.float64))
    L, R, x = rnd(chi, W.shape[0], chi), rnd(chi, W.shape[3], chi), rnd(chi, 2, chi)
    y = torch.empty_like(x)
    nnz = int(np.count_nonzero(W))
    flops = 8.0 * (chi * 2 * chi * (chi * W.shape[0] + chi * W.shape[3]) + chi * chi * nnz)
    st = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(tag, reps=10):
        for _ in range(3):
            g.heff_contract(L, W, R, x, y, prec, stream=st.cuda_stream, env_tag=tag)
        torch.cuda.synchronize()
        a.record(st)
        for _ in range(reps):
            g.heff_contract(L, W, R, x, y, prec, stream=st.cuda_stream, env_tag=tag)
        b.record(st)
        b.synchronize()
        return a.elapsed_time(b) / reps
    return flops, timed(7), timed(None)


def heff_u1_probe(args, g, torch, st, W, mps=None):
    """H_eff applies on the live chi_max state at its centre site (the trajectory's own
    environments and sector structure), CUDA events on the launching stream, environment
    operands cached as in a Lanczos run.  The algorithmic flops are counted over the nonzero
    U(1) blocks (charges read off the state's nonzero pattern) and, for comparison, densely."""
    from paper_2005_06104_gb300 import workloads as wl
    n = len(W)
    dims = st.bond_dims()
    c = max(range(n), key=lambda i: dims[i] * dims[i + 1])
    st.canonicalize(c)
    if mps is None:
        mps = st.get_mps()
    qs = wl.bond_charges(mps[:c + 1])
    cs = wl.mpo_channel_charges(W)
    if any(q is None for q in qs[c]) or any(q is None for q in qs[c + 1]):
        return None
    blocks = wl.heff_flops_u1(qs[c], qs[c + 1], W[c], cs[c], cs[c + 1])
    ml, mr = dims[c], dims[c + 1]
    dense = 8.0 * (ml * 2 * mr * (ml * W[c].shape[0] + mr * W[c].shape[3]) + ml * mr * int(np.count_nonzero(W[c])))
    x = torch.from_numpy(np.ascontiguousarray(mps[c])).cuda()
    y = torch.empty_like(x)
    prec = prec_code(g, args.precision)
    cur = torch.cuda.current_stream()
    for _ in range(3):
        st.heff_apply(c, x, y, prec)
    torch.cuda.synchronize()
    v0, m0 = g.gemm_chunk_stats()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 10
    a.record(cur)
    for _ in range(reps):
        st.heff_apply(c, x, y, prec)
    b.record(cur)
    b.synchronize()
    ms = a.elapsed_time(b) / reps
    v1, m1 = g.gemm_chunk_stats()
    tab_l, tab_r = wl.sector_table(qs[c]), wl.sector_table(qs[c + 1])
    return {"site": c, "ml": ml, "mr": mr, "w": [int(W[c].shape[0]), int(W[c].shape[3])],
            "sectors_left": len(set(qs[c])), "sectors_right": len(set(qs[c + 1])),
            "largest_sector": max(max(d for _, d, _ in tab_l), max(d for _, d, _ in tab_r))
            if tab_l and tab_r else None, "contiguous": tab_l is not None and tab_r is not None,
            "ms_per_apply": ms, "flops_blocks": blocks, "flops_dense": dense, "block_fraction": blocks / dense,
            "tflops_blocks": blocks / ms / 1e9, "tflops_dense_equivalent": dense / ms / 1e9,
            "gemm_chunk_pairs_multiplied": (m1 - m0) / max(1, v1 - v0),
            "timed": f"{reps} applies after 3 warm-up at the centre site of the state after the timed steps"}


def max_over_ranks(x, dist, device):
    """The largest of every rank's x (all ranks receive it)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def job_throughput(world, steps, t_max):
    """Whole-job steps per second: every replica runs `steps` steps; the slowest rank's time counts."""
    return world * steps / t_max


def _pinned_alloc(torch):
    """Page-locked host arrays (numpy views of pinned torch tensors) for the e2e leg."""
    def alloc(shape):
        t = torch.empty(int(np.prod(shape)) * 2, dtype=torch.float64, pin_memory=True)
        return t.numpy().view(np.complex128).reshape(shape)
    return alloc


def comparison_legs(args, g, torch, W, psi0, opts, stream, new_handle, step):
    """Precision form vs FP64 GPU form, and TDVP2 against GSE-TDVP1 (Sec. I.C): one step of
    each from the same state of a second trajectory capped at --compare-chi (an FP64 step at
    chi = 1024 takes tens of minutes)."""
    def timed_step(h, fn):
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea.record()
        fn(h)
        eb.record()
        eb.synchronize()
        return ea.elapsed_time(eb)
    copts = dict(opts, chi_max=args.compare_chi)
    cmp_h = new_handle(psi0, W, stream=stream, **copts)
    for _ in range(args.compare_prep):
        step(cmp_h)
    cmp_state = cmp_h.get_mps()
    cmp_dims = cmp_h.bond_dims()
    cmp_h.close()
    a = new_handle(cmp_state, W, stream=stream, **dict(copts, precision=g.PREC_FP64))
    ms_64 = timed_step(a, step)
    e_64, n_64 = a.energy(), a.norm()
    a.close()
    b_ = new_handle(cmp_state, W, stream=stream, **copts)
    ms_tc = timed_step(b_, step)
    e_tc, n_tc = b_.energy(), b_.norm()
    b_.close()
    prec = {"chi_max": args.compare_chi, "bond_dims_max": max(cmp_dims), "steps_before": args.compare_prep,
            "precision": args.precision, "energy_precision_form": e_tc, "energy_fp64": e_64,
            "step_ms_precision_form": ms_tc, "step_ms_fp64": ms_64, "speedup_over_fp64": ms_64 / ms_tc,
            "rel_energy_err": abs(e_tc - e_64) / abs(e_64), "norm_drift": abs(n_tc - 1.0),
            "norm_drift_fp64": abs(n_64 - 1.0),
            "what": "one GSE-TDVP1 step in each form from the same state of the comparison trajectory"}
    tdvp2 = None
    if not args.no_tdvp2:
        c_ = new_handle(cmp_state, W, stream=stream, **copts)
        c_.trace(True)
        ms_2 = timed_step(c_, lambda h: h.sweep2(args.dt, g.REAL))
        tdvp2 = {"chi_max": args.compare_chi, "step_ms": ms_2, "gse_tdvp1_step_ms": ms_tc,
                 "gse_tdvp1_over_tdvp2": ms_tc / ms_2, "paper_ratio_cpu": 0.36,
                 "bond_dim_max": max(c_.bond_dims()), "energy": c_.energy(),
                 "discarded_weight": c_.trunc_stats()["disc_eps"], "phases_ms": c_.trace_read(),
                 "what": "one TDVP2 step (tdvp_sweep2, same precision form, same cap, eps = 0) and one "
                         "GSE-TDVP1 step from the same state of the comparison trajectory"}
        c_.close()
    return prec, tdvp2


def roofline_line(args, g, torch, W):
    Wmax = max(W, key=lambda w: w.shape[0] * w.shape[3])
    pflops, pms, pms_unc = heff_roofline(g, torch, args.heff_chi, Wmax, prec_code(g, args.precision))
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(peaks_path)) if os.path.exists(peaks_path) else None
    bf16 = peaks["bf16_tflops"] if peaks else 1900.0
    if args.precision.startswith("bf16"):
        # a contraction in BF16 slices: the measured dense BF16 peak; each algorithmic
        # flop costs `products` tensor-core flops
        products = 10 if args.precision == "bf16x10" else 6
        peak, peak_src = bf16, "measured bf16_tflops (MEASURED_PEAKS.json)" if peaks else "fallback 1900 TF/s bf16"
        kern = f"H_eff apply (tcgen05 kind::f16, BF16 exact slices, {products} products) at chi={args.heff_chi}, w=14"
    elif args.precision.startswith("tf32"):
        products = 3
        peak = bf16 * (1.1 / 2.25)  # measured bf16 x nominal tf32/bf16 ratio
        peak_src = "measured bf16_tflops x 1.1/2.25 (nominal tf32/bf16)"
        kern = f"H_eff apply (tcgen05 kind::tf32, 3 split products) at chi={args.heff_chi}, w=14"
    else:
        products, peak, peak_src = 1, 1.097, "cuBLAS DGEMM measured on this part (bench.py --peaks)"
        kern = f"H_eff apply (FP64 CUDA cores) at chi={args.heff_chi}, w=14"
    # DRAM bytes of one apply (its 5 launches), from the ncu capture of these kernels at
    # chi = 1024, w = 14 in BF16X10; other configurations have no capture
    traffic, traffic_src = None, None
    if args.precision == "bf16x10" and args.heff_chi == 1024:
        traffic = 5.121e9
        traffic_src = ("ncu dram__bytes_read.sum + dram__bytes_write.sum over the 5 launches of one cached "
                       "apply (slice x, GEMM 1 with L channel-major, MPO stage, GEMM 3 split 4 ways, split-K "
                       "sum) of these kernels on dense random operands")
    elif args.precision == "bf16x6" and args.heff_chi == 1024:
        traffic = 2.599e9
        traffic_src = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the two k_gemm_bf16s<3> launches of one "
                       "cached apply (1.264 GB GEMM 1, 1.335 GB GEMM 3; 78 % of the apply's device time in the "
                       "launch list); the slicing, MPO-stage and split-K launches are not in this figure")
    achieved = pflops / (pms / 1e3) / 1e12
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic, "kernel": kern, "peak_source": peak_src,
            "traffic_source": traffic_src, "tensor_flops_per_algorithmic_flop": products,
            "tensor_frac_executed": achieved * products / peak, "ms_per_apply": pms,
            "algorithmic_flops_per_apply": pflops, "ms_per_apply_rebuilding_env_operands": pms_unc,
            "timed": "10 applies after 3 warm-up, environment operands cached (as in a Lanczos run)"}


def u1_roofline(dense_roof, u1):
    """The roofline line of the H_eff apply on the U(1) state: achieved = flops over the nonzero
    blocks / measured time; the random dense-operand probe stays as context."""
    u1_traffic = 2.147e9  # DRAM bytes of one apply on U(1) operands of this shape (ncu, see source)
    achieved = u1["tflops_blocks"]
    products = dense_roof["tensor_flops_per_algorithmic_flop"]
    return {"bound": "tensor", "achieved": achieved, "peak": dense_roof["peak"], "unit": "TFLOP/s",
            "frac": achieved / dense_roof["peak"], "traffic": u1_traffic if products == 10 else None,
            "kernel": f"H_eff apply on the chi={max(u1['ml'], u1['mr'])} U(1) state (centre site, w={u1['w']}): "
                      f"slicing, tcgen05 BF16 exact-slice GEMMs ({products} products) skipping all-zero tiles, "
                      "MPO stage",
            "peak_source": dense_roof["peak_source"],
            "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum over the 5 launches of one cached "
                               "BF16X10 apply on U(1) operands of the same shape (charges of the middle bond of a "
                               "24-site random charge-conserving state at bond dimension 1021, the cylinder MPO's "
                               "widest site: bench.py --heff-probe --u1), standing in for the live state"
                               if products == 10 else "no capture for this precision form"),
            "algorithmic_flops": "over the nonzero U(1) blocks (heff_flops_u1)",
            "algorithmic_flops_per_apply": u1["flops_blocks"], "ms_per_apply": u1["ms_per_apply"],
            "tensor_flops_per_algorithmic_flop": products,
            "gemm_chunk_pairs_multiplied": u1["gemm_chunk_pairs_multiplied"],
            "dense_operand_probe": dense_roof}


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
    lat, W, psi0, cfg = workload(args)

    def new_handle(*a, **kw):
        h = g.GseTdvp(*a, **kw)
        if args.krylov == "zipup":
            h.krylov_method(g.KRYLOV_ZIPUP)
        if args.krylov_precision != "same" and kw.get("precision", g.PREC_FP64) != g.PREC_FP64:
            h.krylov_precision(prec_code(g, args.krylov_precision))
        return h
    opts = dict(tau=args.dt, eps_k=1e-8, eps_m=1e-8, eps=0.0, chi_max=args.chi_max,
                precision=prec_code(g, args.precision))
    stream = torch.cuda.current_stream().cuda_stream

    def step(h):
        h.expand_basis(args.k)
        h.sweep(args.dt, g.REAL)

    # bounded legs first (rank 0): the H_eff roofline probe, the CPU oracle sample, the
    # precision-vs-FP64 and TDVP2 comparisons on a trajectory capped at --compare-chi
    legs = {}
    if rank == 0 and not args.step_only:
        legs["roofline"] = roofline_line(args, g, torch, W)
        legs["precision_vs_fp64"], legs["tdvp2_comparison"] = comparison_legs(
            args, g, torch, W, psi0, opts, stream, new_handle, step)
        if not args.no_cpu_baseline:
            try:
                legs["cpu_baseline"] = cpu_baseline(args, W)
            except Exception as ex:  # reported, never silently replaced
                legs["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                        "sample": f"failed: {ex}"}
    # the chi_max trajectory: growth steps, warm-up steps, timed steps
    st = new_handle(psi0, W, stream=stream, **opts)
    e_init = st.energy()
    for _ in range(args.prep_steps + args.warmup):
        step(st)
    start_state = st.get_mps()
    dims_start = st.bond_dims()
    clocks = Clocks(local)
    ts, phases = [], {}
    heff_ms = heff_flops = 0.0
    heff_n = 0
    nfo = {}
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = g.launch_count()
    stopped_early = False
    for i in range(args.steps):
        # time guard: the timed steps left plus the e2e step must fit the wall-clock budget;
        # every rank takes the same decision
        if ts:
            mean_s = sum(ts) / len(ts) / 1e3
            over = (time.time() - T_START) + (args.steps - i + 1) * mean_s > args.time_budget
            if world > 1:
                over = max_over_ranks(1.0 if over else 0.0, dist, "cuda") > 0.0
            if over:
                stopped_early = True
                break
        st.profile(True)
        st.trace(True)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("gse_step")  # lets a profiler select exactly the timed steps
        a.record()
        step(st)
        b.record()
        torch.cuda.nvtx.range_pop()
        b.synchronize()
        ts.append(a.elapsed_time(b))
        pr = st.profile_read()
        for kk, vv in st.trace_read().items():
            phases[kk] = phases.get(kk, 0.0) + vv
        heff_ms += pr["ms"]
        heff_flops += pr["flops"]
        heff_n += pr["applies"]
        nfo = st.trunc_stats()
        nfo["krylov_env_segment"] = st.krylov_memory()
    torch.cuda.synchronize()
    launches = g.launch_count() - launches0
    if world > 1:
        dist.barrier()
    ck = clocks.stop()
    n_timed = len(ts)
    phases = {kk: vv / n_timed for kk, vv in phases.items()}
    t_rank = sum(ts) / 1e3
    if world > 1:
        t_rank = max_over_ranks(t_rank, dist, "cuda")
    value = job_throughput(world, n_timed, t_rank)
    nfo["bond_dim_max"] = max(st.bond_dims())
    nfo["bond_dims_start"] = dims_start
    e_end = st.energy()
    u1 = None
    if rank == 0 and not args.step_only and args.precision != "fp64":
        u1 = heff_u1_probe(args, g, torch, st, W)
    st.close()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    base = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": n_timed,
            "warmup": args.warmup, "ms_per_step": sum(ts) / n_timed, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": f"c128 state / {args.precision} contractions",
            "data": "synthetic", "config": dict(cfg, parallelism=f"replicas{world}", untimed_steps_before=
                                                args.prep_steps + args.warmup),
            "gpu_launches": launches, "clocks": ck, "phases_ms_per_step": phases, "step_stats": nfo}
    if stopped_early:
        base["steps_requested"] = args.steps
        base["stopped_by_time_budget"] = args.time_budget
    if args.step_only:
        print(json.dumps(dict(base, step_only=True)), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return
    # e2e through the public API: the state in page-locked host memory, tdvp_create (copy to the
    # device, canonical form), one step, tdvp_get_mps back into page-locked memory
    alloc = _pinned_alloc(torch)
    host_in = []
    for x in start_state:
        y = alloc(x.shape)
        y[...] = x
        host_in.append(y)
    h2d = sum(x.nbytes for x in host_in) + sum(w.nbytes for w in W)
    torch.cuda.synchronize()
    t = time.perf_counter()
    s2 = new_handle(host_in, W, stream=stream, **opts)
    step(s2)
    out = s2.get_mps(alloc)
    s2.close()
    e2e_s = time.perf_counter() - t
    d2h = sum(x.nbytes for x in out)
    roof = legs.get("roofline")
    if roof is not None and u1 is not None:
        roof = u1_roofline(roof, u1)
    achieved_step = heff_flops / (heff_ms / 1e3) / 1e12 if heff_ms > 0 else None
    line = dict(base)
    line.update({
        "roofline": roof,
        "heff_in_step": {"applies": heff_n / n_timed, "ms": heff_ms / n_timed,
                         "tflops_dense_equivalent": achieved_step,
                         "share_of_step": heff_ms / sum(ts) if ts else None},
        "heff_u1_probe": u1,
        "precision_vs_fp64": legs.get("precision_vs_fp64"),
        "tdvp2_comparison": legs.get("tdvp2_comparison"),
        "energy_conservation": {"E_initial": e_init, "E_after_timed_steps": e_end, "abs_drift": abs(e_end - e_init),
                                "rel_drift": abs(e_end - e_init) / abs(e_init),
                                "steps": args.prep_steps + args.warmup + n_timed},
        "cpu_baseline": legs.get("cpu_baseline"),
        "e2e": {"value": 1.0 / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": 1, "what": "page-locked host MPS -> tdvp_create (copy, canonical form) + expand + sweep "
                                    "+ tdvp_get_mps into page-locked memory + destroy, host wall clock"},
        "wall_s": time.time() - T_START,
    })
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_heff_probe(args):
    import torch
    from paper_2005_06104_gb300 import gse_tdvp as g
    from paper_2005_06104_gb300 import workloads as wl
    Wall = wl.heisenberg_mpo(wl.cylinder_snake(16, 4))
    W = max(Wall, key=lambda w: w.shape[0] * w.shape[3])
    if args.u1:
        # operands with the zero pattern of U(1) charges: the bond charges of the middle of a
        # 24-site random charge-conserving state at bond dimension --heff-chi (sectors sorted),
        # the channel charges of the cylinder MPO's widest site
        i = max(range(len(Wall)), key=lambda j: Wall[j].shape[0] * Wall[j].shape[3])
        cs = wl.mpo_channel_charges(Wall)
        psi = wl.random_u1_mps(24, args.heff_chi, 11, shuffle=False)
        qs = wl.bond_charges(psi)
        L, R, x = wl.u1_heff_operands(qs[12], qs[13], cs[i], cs[i + 1], 5)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        Ld, Rd, xd = dev(L), dev(R), dev(x)
        yd = torch.empty_like(xd)
        prec = prec_code(g, args.precision)
        cur = torch.cuda.current_stream()
        for _ in range(3):
            g.heff_contract(Ld, W, Rd, xd, yd, prec, stream=cur.cuda_stream, env_tag=3)
        torch.cuda.synchronize()
        v0, m0 = g.gemm_chunk_stats()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(cur)
        for _ in range(10):
            g.heff_contract(Ld, W, Rd, xd, yd, prec, stream=cur.cuda_stream, env_tag=3)
        b.record(cur)
        b.synchronize()
        ms = a.elapsed_time(b) / 10
        v1, m1 = g.gemm_chunk_stats()
        blocks = wl.heff_flops_u1(qs[12], qs[13], W, cs[i], cs[i + 1])
        ml, mr = x.shape[0], x.shape[2]
        dense = 8.0 * (ml * 2 * mr * (ml * W.shape[0] + mr * W.shape[3]) + ml * mr * int(np.count_nonzero(W)))
        print(json.dumps({"heff_u1_operands": True, "ml": ml, "mr": mr, "w": int(W.shape[0]),
                          "precision": args.precision, "ms_per_apply": ms, "flops_blocks": blocks,
                          "flops_dense": dense, "tflops_blocks": blocks / ms / 1e9,
                          "gemm_chunk_pairs_multiplied": (m1 - m0) / max(1, v1 - v0)}), flush=True)
        return
    flops, ms, ms_unc = heff_roofline(g, torch, args.heff_chi, W, prec_code(g, args.precision))
    print(json.dumps({"heff_chi": args.heff_chi, "w": int(W.shape[0]), "precision": args.precision,
                      "ms_per_apply": ms, "ms_per_apply_rebuilding_env_operands": ms_unc,
                      "algorithmic_tflops": flops / ms / 1e9}), flush=True)


def run_svd_probe(args):
    """The blocked Jacobi SVD on its own: tdvp_create left-canonicalises a dense random MPS
    of the cylinder's length at bond dimension --heff-chi (no conserved charge, so every
    gauge move is one dense (2m) x m block), timed with CUDA events."""
    import torch
    from paper_2005_06104_gb300 import gse_tdvp as g
    from paper_2005_06104_gb300 import workloads as wl
    lat = wl.cylinder_snake(16, 4)
    W = wl.heisenberg_mpo(lat)
    psi = wl.random_mps(lat.n, args.heff_chi, 3)
    out = []
    for _ in range(2):  # the first call also warms the allocator
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        st = g.GseTdvp(psi, W, stream=torch.cuda.current_stream().cuda_stream)
        b.record()
        b.synchronize()
        out.append(a.elapsed_time(b))
        nfo = st.trunc_stats()
        st.close()
    print(json.dumps({"svd_chi": args.heff_chi, "gauge_moves": lat.n - 1, "ms_create": out[-1],
                      "jacobi_sweeps": nfo["svd_sweeps"], "widest_block": nfo["svd_max_block"]}), flush=True)


def _chain_ground_energy(n):
    """Lowest eigenvalue of the open Heisenberg chain (J = 1, S = sigma/2) in the S^z = 0
    sector, by a sparse Lanczos solver on the basis of bit strings with n/2 up spins."""
    import itertools
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    states = [sum(1 << b for b in c) for c in itertools.combinations(range(n), n // 2)]
    index = {s: i for i, s in enumerate(states)}
    rows, cols, vals = [], [], []
    for i, s in enumerate(states):
        diag = 0.0
        for b in range(n - 1):
            u, v = (s >> b) & 1, (s >> (b + 1)) & 1
            if u == v:
                diag += 0.25
            else:
                diag -= 0.25
                rows.append(index[s ^ (3 << b)])  # S+S- + S-S+ flips the pair, amplitude 1/2
                cols.append(i)
                vals.append(0.5)
        rows.append(i)
        cols.append(i)
        vals.append(diag)
    H = sp.csr_matrix((vals, (rows, cols)), shape=(len(states), len(states)))
    return float(spla.eigsh(H, k=1, which="SA", tol=1e-12)[0][0])


def run_fig3(args):
    """Imaginary time on the rung-decoupled zigzag ladder from Neel (Sec. II.A, Fig. 3 at leg
    length --fig3-leg): GSE-TDVP1 at d tau = 0.1 and 0.4 (i tau = 1/lambda, k = 3,
    eps_K = 1e-12, eps_M = 1e-8, eps = 1e-10, chi_max 128) against twice the exact ground
    energy of one leg, and TDVP2 from the same product state."""
    import torch
    from paper_2005_06104_gb300 import gse_tdvp as g
    from paper_2005_06104_gb300 import workloads as wl
    lx = args.fig3_leg
    lat = wl.zigzag_ladder(lx, 1.0, 0.0)
    W = wl.heisenberg_mpo(lat)
    lam = wl.lambda_top(lat)
    e_ref = 2.0 * _chain_ground_energy(lx)
    kw = dict(tau=-1j / lam, eps_k=1e-12, eps_m=1e-8, eps=1e-10, chi_max=128,
              stream=torch.cuda.current_stream().cuda_stream)
    out = {"leg": lx, "n_sites": lat.n, "E_ref": e_ref, "tau_max": args.fig3_tau, "runs": {}}
    for dt in (0.1, 0.4):
        st = g.GseTdvp(wl.neel_state(lat), W, **kw)
        trace = []
        for step in range(1, int(round(args.fig3_tau / dt)) + 1):
            st.step(dt, g.IMAG, 3)
            e = st.energy()
            trace.append([round(step * dt, 6), e, (e - e_ref) / abs(e_ref), max(st.bond_dims())])
        st.close()
        out["runs"][f"gse_tdvp1_dt{dt}"] = trace
    st = g.GseTdvp(wl.neel_state(lat), W, **kw)
    e0 = st.energy()
    trace = []
    for step in range(1, 6):
        st.sweep2(0.1, g.IMAG)
        e = st.energy()
        trace.append([round(step * 0.1, 6), e, (e - e_ref) / abs(e_ref), max(st.bond_dims())])
    st.close()
    out["runs"]["tdvp2_dt0.1"] = trace
    out["E_neel"] = e0
    print(json.dumps(out), flush=True)


def run_config2(args):
    """Rung-decoupled 2 x 20 zigzag ladder from a random product state (seed 1), imaginary time
    d tau = 0.1, k = 3, i tau = 1/lambda, eps_K = 1e-12, eps_M = 1e-8, eps = 1e-10, chi <= 128,
    50 steps (Sec. II.A setting at leg 20), in FP64, TF32X3 and BF16X10: energies per step
    against twice the exact ground energy of one 20-site leg (sparse Lanczos in S^z = 0)."""
    import torch
    from paper_2005_06104_gb300 import gse_tdvp as g
    from paper_2005_06104_gb300 import workloads as wl
    p = wl.workload("ladder2x20_rd")
    lat, W, psi = p["lattice"], p["mpo"], p["psi"]
    e_ref = 2.0 * _chain_ground_energy(20)
    stream = torch.cuda.current_stream().cuda_stream
    kw = dict(tau=p["tau"], eps_k=p["eps_k"], eps_m=p["eps_m"], eps=p["eps"], chi_max=p["chi_max"], stream=stream)
    runs = {}
    for name in ("fp64", "tf32x3", "bf16x10"):
        st = g.GseTdvp(psi, W, precision=prec_code(g, name), **kw)
        es, dims = [], []
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(p["steps"]):
            st.step(p["dt"], g.IMAG, p["k"])
            es.append(st.energy())
            dims.append(max(st.bond_dims()))
        el = time.perf_counter() - t
        st.close()
        runs[name] = {"energies": es, "bond_dim_max": dims, "s_per_step": el / p["steps"]}
    e64 = runs["fp64"]["energies"]
    out = {"config": "ladder2x20_rd", "steps": p["steps"], "E_ref_2E0_L20": e_ref,
           "final_rel_err_vs_2E0": {k: (v["energies"][-1] - e_ref) / abs(e_ref) for k, v in runs.items()},
           "monotone_non_increasing": {k: all(b <= a + 1e-12 for a, b in zip(v["energies"], v["energies"][1:]))
                                       for k, v in runs.items()},
           "max_rel_diff_vs_fp64": {k: max(abs(a - b) / abs(b) for a, b in zip(v["energies"], e64))
                                    for k, v in runs.items() if k != "fp64"},
           "bond_dim_max_final": {k: v["bond_dim_max"][-1] for k, v in runs.items()},
           "s_per_step": {k: v["s_per_step"] for k, v in runs.items()},
           "energies_fp64": e64}
    print(json.dumps(out), flush=True)


def run_config3(args):
    """Rung-coupled 2 x 50 zigzag ladder, Neel with the spin at (25, 0) flipped, real time dt = 0.1,
    k = 3, chi <= 512, 40 steps in BF16X10.  At steps 1, 10, 20, 30, 40 the state is copied
    and one FP64 step and one precision-form step run from it: per-step relative energy error
    and norm drift of the precision form against FP64."""
    import torch
    from paper_2005_06104_gb300 import gse_tdvp as g
    from paper_2005_06104_gb300 import workloads as wl
    p = wl.workload("ladder2x50")
    W, psi = p["mpo"], p["psi"]
    stream = torch.cuda.current_stream().cuda_stream
    kw = dict(tau=p["tau"], eps_k=p["eps_k"], eps_m=p["eps_m"], eps=p["eps"], chi_max=p["chi_max"], stream=stream)
    st = g.GseTdvp(psi, W, precision=g.PREC_BF16X10, **kw)
    e0 = st.energy()
    checks, es, dims, ts = [], [], [], []
    for step in range(1, p["steps"] + 1):
        torch.cuda.synchronize()
        t = time.perf_counter()
        st.step(p["dt"], g.REAL, p["k"])
        ts.append(time.perf_counter() - t)
        es.append(st.energy())
        dims.append(max(st.bond_dims()))
        if step in (1, 10, 20, 30, 40):
            state = st.get_mps()
            a = g.GseTdvp(state, W, precision=g.PREC_FP64, **kw)
            b = g.GseTdvp(state, W, precision=g.PREC_BF16X10, **kw)
            a.step(p["dt"], g.REAL, p["k"])
            b.step(p["dt"], g.REAL, p["k"])
            ea, eb = a.energy(), b.energy()
            checks.append({"after_step": step, "bond_dim_max": dims[-1], "rel_energy_err": abs(eb - ea) / abs(ea),
                           "norm_drift": abs(b.norm() - 1.0), "norm_drift_fp64": abs(a.norm() - 1.0)})
            a.close()
            b.close()
    st.close()
    print(json.dumps({"config": "ladder2x50", "steps": p["steps"], "chi_max": p["chi_max"], "E0": e0,
                      "energy_drift_abs": abs(es[-1] - e0), "energy_drift_rel": abs(es[-1] - e0) / abs(e0),
                      "per_step_checks": checks, "bond_dim_max": dims, "s_per_step": ts}), flush=True)


def run_oat(args):
    """One-axis twisting at the paper's size (Sec. II.B, Fig. 4 setting): N = 100, H = (S^z)^2
    (w = 3), all spins along +x, real time to t = 0.25, eps = 0; GSE-TDVP1 at dt = 0.025 (k = 3,
    eps_K = eps_M = 1e-4) and dt = 0.05 (k = 5, eps_K = 1e-4, eps_M = 1e-8), TDVP2 at dt = 0.025
    (eps = 1e-7), all capped at --oat-chi, FP64.  <S^x> and xi^2 (Eqs. 13-15, from MPO
    expectations of total-spin products) against the exact Dicke-subspace solution; relative
    energy error; bond dimensions."""
    import torch
    from oracle import oat_exact as X
    from paper_2005_06104_gb300 import gse_tdvp as g
    from paper_2005_06104_gb300 import workloads as wl
    n = 100
    W = wl.oat_mpo(n)
    Mx, My, Mz = (wl.total_op_mpo(n, op) for op in (wl.SX, wl.SY, wl.SZ))
    ops = {"x": Mx, "yy": wl.mpo_product(My, My), "zz": wl.mpo_product(Mz, Mz), "yz": wl.mpo_product(My, Mz),
           "zy": wl.mpo_product(Mz, My)}
    stream = torch.cuda.current_stream().cuda_stream
    runs = {}
    settings = [("gse_tdvp1_dt0.025_k3", 0.025, 3, 1e-4, 1e-4, 0.0, False),
                ("gse_tdvp1_dt0.05_k5", 0.05, 5, 1e-4, 1e-8, 0.0, False),
                ("tdvp2_dt0.025_eps1e-7", 0.025, 1, 1e-4, 1e-4, 1e-7, True)]
    for name, dt, k, ek, em, eps, two in settings:
        st = g.GseTdvp(wl.x_polarized_state(n), W, tau=dt, eps_k=ek, eps_m=em, eps=eps, chi_max=args.oat_chi,
                       lanczos_max=63, stream=stream)
        e0 = st.energy()
        rows = []
        t0 = time.perf_counter()
        for step in range(1, int(round(0.25 / dt)) + 1):
            if two:
                st.sweep2(dt, g.REAL)
            else:
                st.step(dt, g.REAL, k)
            mom = {kk: st.expect_mpo(v) for kk, v in ops.items()}
            ex = X.oat_moments(n, step * dt)
            rows.append({"t": round(step * dt, 6), "sx": mom["x"].real, "sx_exact": ex["x"].real,
                         "xi2": X.squeezing_xi2(mom, n), "xi2_exact": X.squeezing_xi2(ex, n),
                         "rel_energy_err": abs(st.energy() - e0) / abs(e0), "bond_dim_max": max(st.bond_dims())})
        runs[name] = {"s_total": time.perf_counter() - t0, "trajectory": rows}
        st.close()
    print(json.dumps({"workload": "oat_n100_x_polarized", "chi_max": args.oat_chi, "runs": runs}), flush=True)


def run_peaks(args):
    """Library matmul peaks of the arithmetic the FP64 factorisations, the FP32 Jacobi rotations
    and the TF32 form run in (the measured BF16 peak and the copy bandwidth come with the
    machine): torch.matmul (cuBLAS) on n x n operands, best of 5 timed with CUDA events after
    2 warm-ups, 2 n^3 flops per real product."""
    import torch
    out = {}
    for name, dtype, tf32 in [("fp64", torch.float64, False), ("fp32_simt", torch.float32, False),
                              ("tf32", torch.float32, True), ("c128_zgemm", torch.complex128, False)]:
        torch.backends.cuda.matmul.allow_tf32 = tf32
        n = 4096 if dtype in (torch.float64, torch.complex128) else 8192
        a = torch.randn(n, n, device="cuda", dtype=dtype)
        b = torch.randn(n, n, device="cuda", dtype=dtype)
        for _ in range(2):
            torch.matmul(a, b)
        best = None
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        flops = (8.0 if dtype == torch.complex128 else 2.0) * n ** 3
        out[name] = {"n": n, "ms": best, "tflops": flops / best / 1e9}
    torch.backends.cuda.matmul.allow_tf32 = False
    print(json.dumps({"peaks": out, "how": "torch.matmul best of 5 (CUDA events), 2 n^3 real flops, 8 n^3 complex"}),
          flush=True)


def run_batch(args):
    """Independent random-field chains stepped as one batch (one stream per chain, host worker
    pool) against the same chains stepped one after another on one stream each, same steps."""
    import torch
    from paper_2005_06104_gb300 import gse_tdvp as g
    from paper_2005_06104_gb300 import workloads as wl
    torch.cuda.set_device(0)
    spec = wl.random_field_chains(args.batch_chains, seed=0)
    chains = [(c["psi"], c["mpo"], dict(tau=c["tau"], eps_k=1e-8, eps_m=1e-8, chi_max=c["chi_max"],
                                        precision=prec_code(g, args.precision))) for c in spec]
    dt, k = spec[0]["dt"], spec[0]["k"]

    def timed(n_threads):
        b = g.GseTdvpBatch(chains, n_threads=n_threads)
        for _ in range(args.prep_steps + args.warmup):
            b.step(dt, g.REAL, k)
        torch.cuda.synchronize()
        l0 = g.launch_count()
        t = time.perf_counter()
        for _ in range(args.steps):
            b.step(dt, g.REAL, k)
        torch.cuda.synchronize()
        el = time.perf_counter() - t
        dims = [max(b.chain(i).bond_dims()) for i in range(len(chains))]
        e = b.energies()
        b.close()
        return el, g.launch_count() - l0, dims, e

    t_b, l_b, dims, e_b = timed(args.batch_threads)
    t_1, _, _, e_1 = timed(1)
    n = len(chains)
    print(json.dumps({
        "metric": "GSE-TDVP1 chain steps/s, batch of independent random-field chains", "unit": "chain steps/s",
        "value": n * args.steps / t_b, "sequential_value": n * args.steps / t_1, "speedup": t_1 / t_b,
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "prep_steps": args.prep_steps,
        "higher_is_better": True, "dtype": f"c128 state / {args.precision} contractions", "data": "synthetic",
        "config": {"workload": f"random_field_heisenberg_chains_{n}", "lengths": "U{20..60}", "fields": "U[-2,2]",
                   "chi_max": "U{32..128}", "dt": dt, "k": k, "seed": 0, "start": "Neel",
                   "batch_threads": args.batch_threads or os.cpu_count()},
        "gpu_launches": l_b, "bond_dim_max_per_chain": dims,
        "max_energy_difference_batch_vs_sequential": max(abs(a - b) for a, b in zip(e_b, e_1)),
        "timing": "host wall clock around the timed batch steps, synchronised on both sides"}), flush=True)


def main():
    args = parse()
    if args.batch_chains > 0:
        run_batch(args)
        return
    if args.peaks:
        run_peaks(args)
    elif args.oat:
        run_oat(args)
    elif args.config2:
        run_config2(args)
    elif args.config3:
        run_config3(args)
    elif args.fig3:
        run_fig3(args)
    elif args.svd_probe:
        run_svd_probe(args)
    elif args.heff_probe:
        run_heff_probe(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
