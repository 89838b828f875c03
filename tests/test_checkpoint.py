"""Checkpoint files (host-only C entry points): round trip, and every corruption is refused."""
import os

import numpy as np
import pytest

from paper_2005_06104_gb300 import workloads as wl


@pytest.fixture(scope="module")
def g():
    from paper_2005_06104_gb300 import build
    if not os.path.exists(os.path.join(os.path.dirname(build.__file__), "libgsetdvp.so")):
        build.build()
    from paper_2005_06104_gb300 import gse_tdvp
    return gse_tdvp


def test_round_trip_is_bit_exact(g, tmp_path):
    psi = wl.random_mps(9, 7, 3)
    p = tmp_path / "state.gse"
    g.write_checkpoint(p, psi)
    n, d, m = g.checkpoint_header(p)
    assert (n, d, m) == (9, 2, wl.mps_bond_dims(psi))
    back = g.read_checkpoint(p)
    assert all(np.array_equal(a, b) for a, b in zip(psi, back))
    assert not os.path.exists(str(p) + ".tmp")


def test_overwrite_replaces_the_file(g, tmp_path):
    p = tmp_path / "state.gse"
    g.write_checkpoint(p, wl.random_mps(4, 3, 1))
    psi = wl.random_mps(5, 4, 2)
    g.write_checkpoint(p, psi)
    assert all(np.array_equal(a, b) for a, b in zip(psi, g.read_checkpoint(p)))


@pytest.mark.parametrize("where", ["magic", "payload", "hash", "truncate"])
def test_corruption_is_refused(g, tmp_path, where):
    p = tmp_path / "state.gse"
    g.write_checkpoint(p, wl.random_mps(6, 5, 4))
    raw = bytearray(p.read_bytes())
    if where == "magic":
        raw[0] ^= 0x20
    elif where == "payload":
        raw[len(raw) // 2] ^= 0x01
    elif where == "hash":
        raw[-1] ^= 0x80
    else:
        raw = raw[:-9]
    p.write_bytes(bytes(raw))
    with pytest.raises(g.TDVPError) as e:
        g.read_checkpoint(p)
    assert e.value.status == 1


def test_inconsistent_dimensions_are_refused(g, tmp_path):
    bad = [np.zeros((2, 2, 3), complex), np.zeros((3, 2, 1), complex)]  # m_0 must be 1
    with pytest.raises(g.TDVPError) as e:
        g.write_checkpoint(tmp_path / "x.gse", bad)
    assert e.value.status == 2
    with pytest.raises(g.TDVPError):
        g.read_checkpoint(tmp_path / "missing.gse")
