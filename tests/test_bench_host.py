"""Host-side pieces of the benchmark that need no GPU: the oracle's CPU baseline sample and
the reference arm's JSON line."""
import argparse
import json
import subprocess
import sys
import os

import pytest

import bench
from paper_2005_06104_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_cpu_baseline_sample_is_bounded_and_scaled():
    lat = wl.cylinder_snake(16, 4)
    W = wl.heisenberg_mpo(lat)
    a = argparse.Namespace(chi_max=32, dt=0.1)
    iters = bench._lanczos_iters_oracle(a, W, chi=8)
    assert 2.0 <= iters <= 40.0
    r = bench.cpu_baseline(a, W, iters)
    assert r["kind"].startswith("oracle") and "extrapolated" in r["kind"]
    assert r["unit"] == bench.UNIT and r["value"] > 0 and r["sample_s"] > 0
    # one sweep = 2N site updates weighted by m_l m_r (m_l + m_r); the centre has the largest share
    assert 1.0 / r["value"] >= 2.0 * r["seconds_per_site_update"]
    assert "chi=32" in r["sample"]


def test_reference_arm_prints_one_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1", "--chi-max", "32"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["value"] == line["value"]
    assert line["config"]["chi_max"] == 32
    # ms_per_step is the measured sample time; the extrapolated sweep time is reported beside it
    assert line["ms_per_step"] == pytest.approx(1e3 * line["cpu_baseline"]["sample_s"], rel=1e-9)
    assert line["extrapolated_ms_per_sweep"] == pytest.approx(1e3 / line["value"], rel=1e-9)


@pytest.mark.parametrize("n", [6, 8, 10])
def test_fig3_reference_energy_matches_dense_ed(n):
    """The --fig3 reference (sparse S^z = 0 Lanczos written from the bond terms) equals the
    Kronecker-product Hamiltonian's ground energy in that sector."""
    from exact import ground_energy_sz0
    ref = ground_energy_sz0(n, [(i, i + 1, 1.0) for i in range(n - 1)])
    assert abs(bench._chain_ground_energy(n) - ref) < 1e-12


def test_u1_roofline_object_follows_the_block_count():
    """The roofline object of the line: achieved is the H_eff flops over the nonzero blocks per
    measured apply, frac = achieved / peak, the dense-operand probe kept beside it; job
    throughput counts every replica's steps against the slowest rank's time."""
    dense = {"tensor_flops_per_algorithmic_flop": 10, "peak": 1903.1, "peak_source": "measured",
             "achieved": 106.0, "frac": 106.0 / 1903.1}
    u1 = {"tflops_blocks": 15.0, "ml": 1024, "mr": 1020, "w": [14, 14], "flops_blocks": 2.52e10,
          "ms_per_apply": 1.68, "gemm_chunk_pairs_multiplied": 0.216}
    r = bench.u1_roofline(dense, u1)
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in r
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["frac"] == pytest.approx(15.0 / 1903.1)
    assert r["traffic"] > 0 and r["dense_operand_probe"] is dense
    assert bench.u1_roofline(dict(dense, tensor_flops_per_algorithmic_flop=6), u1)["traffic"] is None
    assert bench.job_throughput(4, 20, 10.0) == pytest.approx(8.0)


@pytest.mark.parametrize("prec", ["bf16x10", "bf16x6", "tf32x3", "fp64"])
def test_roofline_line_assembles_for_every_precision(monkeypatch, prec):
    """The dense-operand roofline object (the probe's timing replaced by fixed numbers): peaks
    and traffic sources per precision form, frac = achieved / peak."""
    monkeypatch.setattr(bench, "heff_roofline", lambda g, torch, chi, W, p: (4.813e11, 4.5, 5.1))
    g = argparse.Namespace(**{v: i for i, v in enumerate(bench.PRECISIONS.values())})
    W = wl.heisenberg_mpo(wl.cylinder_snake(16, 4))
    a = argparse.Namespace(precision=prec, heff_chi=1024)
    r = bench.roofline_line(a, g, None, W)
    assert r["achieved"] == pytest.approx(4.813e11 / 4.5e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert (r["traffic"] is not None) == (prec in ("bf16x10", "bf16x6"))
    assert r["tensor_flops_per_algorithmic_flop"] == {"bf16x10": 10, "bf16x6": 6, "tf32x3": 3, "fp64": 1}[prec]
