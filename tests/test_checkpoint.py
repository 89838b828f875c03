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


def _rewrite_header(raw, n=None, dims=None):
    """Returns raw with its N field and/or bond dimensions replaced (hash left stale)."""
    import struct
    raw = bytearray(raw)
    if n is not None:
        raw[12:16] = struct.pack("<i", n)
    if dims is not None:
        for i, m in enumerate(dims):
            raw[24 + 4 * i:28 + 4 * i] = struct.pack("<i", m)
    return bytes(raw)


def test_oversized_header_is_refused_before_allocating(g, tmp_path):
    """A header that claims huge bond dimensions (about 2^40 doubles) in a small file: refused
    by the size check, before any buffer of that size exists."""
    psi = wl.random_mps(4, 3, 5)
    p = tmp_path / "big.gse"
    g.write_checkpoint(p, psi)
    m = wl.mps_bond_dims(psi)
    big = [1, 1 << 20, 1 << 20, 1 << 20, 1]
    p.write_bytes(_rewrite_header(p.read_bytes(), dims=big))
    assert g.checkpoint_header(p)[2] == big            # the header alone is well-formed
    arrs = [np.empty((m[i], 2, m[i + 1]), complex) for i in range(4)]
    import ctypes as C
    ptrs = (C.c_void_p * 4)(*[a.ctypes.data for a in arrs])
    dims = (C.c_int * 5)(*big)
    st = g._lib.tdvp_checkpoint_read(str(p).encode(), 4, 2, C.cast(dims, C.c_void_p), ptrs)
    assert st == 1 and b"size" in g._lib.tdvp_checkpoint_last_error()
    with pytest.raises(g.TDVPError) as e:
        g.GseTdvp.load(p, wl.heisenberg_mpo(wl.chain(4)))
    assert e.value.status == 1


def test_buffers_of_other_shapes_are_never_written(g, tmp_path):
    """The caller states its buffers' shapes; a file whose dimensions changed since the header
    was read (here: another state saved under the same name) is refused, buffers untouched."""
    p = tmp_path / "state.gse"
    g.write_checkpoint(p, wl.random_mps(5, 3, 1))
    n, d, m = g.checkpoint_header(p)
    arrs = [np.full((m[i], d, m[i + 1]), 7.0 + 0j) for i in range(n)]
    g.write_checkpoint(p, wl.random_mps(5, 4, 2))      # replaced between header and read
    import ctypes as C
    ptrs = (C.c_void_p * n)(*[a.ctypes.data for a in arrs])
    dims = (C.c_int * (n + 1))(*m)
    st = g._lib.tdvp_checkpoint_read(str(p).encode(), n, d, C.cast(dims, C.c_void_p), ptrs)
    assert st == 2
    assert all(np.all(a == 7.0) for a in arrs)
    # too small a bond_dims buffer for the header
    small = (C.c_int * 2)()
    nn, dd = C.c_int(0), C.c_int(0)
    st = g._lib.tdvp_checkpoint_read_header(str(p).encode(), C.byref(nn), C.byref(dd), C.cast(small, C.c_void_p), 2)
    assert st == 2 and list(small) == [0, 0]


@pytest.mark.parametrize("cut", [1, 20, 200])
def test_load_refuses_truncated_files(g, tmp_path, cut):
    """tdvp_load reads and verifies the whole file before it creates anything on the device."""
    p = tmp_path / "state.gse"
    g.write_checkpoint(p, wl.random_mps(6, 4, 3))
    raw = p.read_bytes()
    p.write_bytes(raw[:-cut])
    with pytest.raises(g.TDVPError) as e:
        g.GseTdvp.load(p, wl.heisenberg_mpo(wl.chain(6)))
    assert e.value.status == 1
