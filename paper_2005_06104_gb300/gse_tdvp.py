"""Python binding of libgsetdvp.so (C ABI in include/gse_tdvp.h).

Argument marshalling only: every step of GSE-TDVP1 runs in the CUDA library.
Device buffers are torch CUDA tensors (complex128), host tensors numpy arrays.
Importing this module loads the library and raises ImportError when it has
not been built (`python -m paper_2005_06104_gb300.build` or
`__graft_entry__.build()`); there is no other implementation to fall back to.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgsetdvp.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "gse_tdvp.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first")
_lib = C.CDLL(LIB_PATH)

REAL, IMAG = 0, 1
PREC_FP64, PREC_TF32X3, PREC_TF32X3_ENV, PREC_BF16X10, PREC_BF16X6 = 0, 1, 2, 3, 4
KRYLOV_DENSITY_MATRIX, KRYLOV_ZIPUP = 0, 1
STATUS = {0: "ok", 1: "invalid argument", 2: "shape mismatch", 3: "out of memory",
          4: "Lanczos not converged", 5: "non-finite value", 6: "device wait timed out",
          7: "CUDA error", 8: "SVD not converged"}


class TDVPError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Options(C.Structure):
    _fields_ = [("tau_re", C.c_double), ("tau_im", C.c_double), ("eps_k", C.c_double),
                ("eps_m", C.c_double), ("eps", C.c_double), ("chi_max", C.c_int),
                ("lanczos_tol", C.c_double), ("lanczos_max", C.c_int), ("precision", C.c_int)]


class _Desc(C.Structure):
    _fields_ = [("n_sites", C.c_int), ("d", C.c_int), ("bond_dims", C.POINTER(C.c_int)),
                ("sites", C.POINTER(C.c_void_p))]


_h = C.c_void_p
_sig = {
    "tdvp_default_options": [C.POINTER(Options)],
    "tdvp_create": [C.POINTER(_Desc), C.POINTER(_Desc), C.POINTER(Options), C.c_void_p, C.POINTER(_h)],
    "tdvp_destroy": [_h],
    "tdvp_set_options": [_h, C.POINTER(Options)],
    "tdvp_canonicalize": [_h, C.c_int],
    "tdvp_expand_basis": [_h, C.c_int, C.c_void_p],
    "tdvp_apply_krylov": [_h],
    "tdvp_sweep": [_h, C.c_double, C.c_int],
    "tdvp_sweep2": [_h, C.c_double, C.c_int],
    "tdvp_krylov_memory": [_h, C.c_double, C.POINTER(C.c_int)],
    "tdvp_set_krylov_method": [_h, C.c_int],
    "tdvp_set_krylov_precision": [_h, C.c_int],
    "tdvp_heff_apply": [_h, C.c_int, C.c_void_p, C.c_void_p, C.c_int],
    "tdvp_keff_apply": [_h, C.c_int, C.c_void_p, C.c_void_p, C.c_int],
    "tdvp_evolve_site": [_h, C.c_int, C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.c_int,
                         C.POINTER(C.c_int)],
    "tdvp_energy": [_h, C.POINTER(C.c_double)],
    "tdvp_norm": [_h, C.POINTER(C.c_double)],
    "tdvp_expect_local": [_h, C.c_void_p, C.c_int, C.POINTER(C.c_double)],
    "tdvp_expect_mpo": [_h, C.POINTER(_Desc), C.POINTER(C.c_double)],
    "tdvp_bond_dims": [_h, C.POINTER(C.c_int)],
    "tdvp_center": [_h, C.POINTER(C.c_int)],
    "tdvp_bond_charges": [_h, C.POINTER(C.c_int), C.POINTER(C.c_int)],
    "tdvp_bond_sectors": [_h, C.POINTER(C.c_int), C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                          C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)],
    "tdvp_trunc_stats": [_h, C.POINTER(C.c_double)],
    "tdvp_get_mps": [_h, C.POINTER(C.c_void_p)],
    "tdvp_profile": [_h, C.c_int],
    "tdvp_profile_read": [_h, C.POINTER(C.c_double)],
    "tdvp_trace": [_h, C.c_int],
    "tdvp_trace_read": [_h, C.POINTER(C.c_double), C.c_int],
}
for _name, _args in _sig.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = C.c_int
_lib.tdvp_last_error.argtypes = [_h]
_lib.tdvp_last_error.restype = C.c_char_p
_lib.tdvp_status_string.argtypes = [C.c_int]
_lib.tdvp_status_string.restype = C.c_char_p
_lib.tdvp_contract_last_error.argtypes = []
_lib.tdvp_contract_last_error.restype = C.c_char_p
_lib.tdvp_launch_count.argtypes = [C.POINTER(C.c_longlong)]
_lib.tdvp_launch_count.restype = C.c_int


def launch_count():
    """Kernels the library has launched in this process (all handles and calls)."""
    out = C.c_longlong(0)
    s = _lib.tdvp_launch_count(C.byref(out))
    if s != 0:
        raise TDVPError(s, "tdvp_launch_count")
    return out.value


_lib.tdvp_gemm_chunk_stats.argtypes = [C.POINTER(C.c_longlong)]
_lib.tdvp_gemm_chunk_stats.restype = C.c_int


def gemm_chunk_stats():
    """(visited, multiplied): (output tile, K chunk) pairs of the BF16 tensor-core GEMMs on the
    current device since load; the difference is the all-zero block work that was skipped."""
    out = (C.c_longlong * 2)()
    s = _lib.tdvp_gemm_chunk_stats(out)
    if s != 0:
        raise TDVPError(s, "tdvp_gemm_chunk_stats")
    return int(out[0]), int(out[1])


class SiteDims(C.Structure):
    _fields_ = [("ml", C.c_int), ("mr", C.c_int), ("wl", C.c_int), ("wr", C.c_int), ("d", C.c_int)]


_raw = {
    "tdvp_heff_contract": [C.POINTER(SiteDims), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                           C.c_int, C.c_void_p],
    "tdvp_heff_contract_cached": [C.POINTER(SiteDims), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_int, C.c_longlong, C.c_void_p],
    "tdvp_keff_contract": [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "tdvp_env_contract": [C.POINTER(SiteDims), C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                          C.c_void_p],
    "tdvp_expm_contract": [C.POINTER(SiteDims), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                           C.c_double, C.c_int, C.c_int, C.c_double, C.c_int, C.POINTER(C.c_int), C.c_void_p],
}
for _name, _args in _raw.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = C.c_int


def _raw_chk(s):
    if s != 0:
        raise TDVPError(s, _lib.tdvp_contract_last_error().decode())


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _host(w):
    w = np.ascontiguousarray(w, dtype=np.complex128)
    return w, C.c_void_p(w.ctypes.data)


def _stream(stream):
    return C.c_void_p(stream or 0)


def _check_site_args(L, W, R, x, y):
    """Shapes, dtype and placement of the operands of one H_eff contraction; returns
    (ml, mr, wl, wr, d).  L [ml, wl, ml], R [mr, wr, mr], x and y [ml, d, mr]: contiguous CUDA
    complex128 tensors; W host [wl, d, d, wr]."""
    ml, wl, ml2 = L.shape
    mr, wr, mr2 = R.shape
    d = W.shape[1]
    if ml2 != ml or mr2 != mr or W.shape != (wl, d, d, wr):
        raise ValueError(f"H_eff operands: L {tuple(L.shape)}, W {W.shape}, R {tuple(R.shape)} do not fit")
    for name, t in (("x", x), ("y", y)):
        if tuple(t.shape) != (ml, d, mr):
            raise ValueError(f"H_eff operands: {name} has shape {tuple(t.shape)}, expected {(ml, d, mr)}")
    for name, t in (("L", L), ("R", R), ("x", x), ("y", y)):
        if not (t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch.complex128"):
            raise ValueError(f"H_eff operands: {name} must be a contiguous CUDA complex128 tensor")
    return ml, mr, wl, wr, d


def heff_contract(L, W, R, x, y, precision=PREC_FP64, stream=None, env_tag=None):
    """y = H_eff x on caller tensors: L, R, x, y torch CUDA complex128; W numpy [wl, d, d, wr].
    env_tag (int >= 0): reuse the tensor-core operand forms of L and R across calls with
    the same tag (the caller guarantees L, R, W unchanged)."""
    ml, mr, wl, wr, d = _check_site_args(L, W, R, x, y)
    Wc, wp = _host(W)
    dims = C.byref(SiteDims(ml, mr, wl, wr, d))
    if env_tag is None:
        _raw_chk(_lib.tdvp_heff_contract(dims, _ptr(L), wp, _ptr(R), _ptr(x), _ptr(y), precision, _stream(stream)))
    else:
        _raw_chk(_lib.tdvp_heff_contract_cached(dims, _ptr(L), wp, _ptr(R), _ptr(x), _ptr(y), precision,
                                                int(env_tag), _stream(stream)))


def _check_dev(**ts):
    """name=(tensor, expected shape): contiguous CUDA complex128 tensors of those shapes."""
    for name, (t, shape) in ts.items():
        if tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
        if not (t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch.complex128"):
            raise ValueError(f"{name} must be a contiguous CUDA complex128 tensor")


def keff_contract(L, R, x, y, stream=None):
    """y[a, c] = sum L[a, w, a'] x[a', b'] R[c, w, b'] on caller tensors: L [ml, w, ml],
    R [mr, w, mr], x and y [ml, mr] (CUDA complex128)."""
    ml, w, _ = L.shape
    mr = R.shape[0]
    _check_dev(L=(L, (ml, w, ml)), R=(R, (mr, w, mr)), x=(x, (ml, mr)), y=(y, (ml, mr)))
    _raw_chk(_lib.tdvp_keff_contract(ml, mr, w, _ptr(L), _ptr(R), _ptr(x), _ptr(y), _stream(stream)))


def env_contract(side, E, W, A, out, stream=None):
    """side 0: left environment update through site A (E = L [ml, wl, ml] -> out [mr, wr, mr]);
    side 1: right environment update (E = R [mr, wr, mr] -> out [ml, wl, ml]).  A [ml, d, mr],
    W host [wl, d, d, wr]."""
    ml, d, mr = A.shape
    wl, wr = W.shape[0], W.shape[3]
    if W.shape != (wl, d, d, wr):
        raise ValueError(f"env_contract: W {W.shape} does not fit A {tuple(A.shape)}")
    if side in (0, 1):
        e_shape, o_shape = ((ml, wl, ml), (mr, wr, mr)) if side == 0 else ((mr, wr, mr), (ml, wl, ml))
        _check_dev(E=(E, e_shape), A=(A, (ml, d, mr)), out=(out, o_shape))
    Wc, wp = _host(W)
    _raw_chk(_lib.tdvp_env_contract(C.byref(SiteDims(ml, mr, wl, wr, d)), side, _ptr(E), wp, _ptr(A), _ptr(out),
                                    _stream(stream)))


def expm_contract(L, W, R, x, y, delta, kind=REAL, precision=PREC_FP64, tol=1e-12, nmax=40, stream=None):
    """y = exp(-i delta H_eff) x (REAL) or exp(-delta H_eff) x (IMAG) on caller tensors, shapes as
    heff_contract; returns the Krylov dimension used."""
    ml, mr, wl, wr, d = _check_site_args(L, W, R, x, y)
    Wc, wp = _host(W)
    it = C.c_int(0)
    _raw_chk(_lib.tdvp_expm_contract(C.byref(SiteDims(ml, mr, wl, wr, d)), _ptr(L), wp, _ptr(R), _ptr(x), _ptr(y),
                                     delta, kind, precision, tol, nmax, C.byref(it), _stream(stream)))
    return it.value


_lib.tdvp_heff_contract_noalloc.argtypes = [C.POINTER(SiteDims), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                             C.c_void_p, C.c_void_p, C.c_char_p, C.c_int]
_lib.tdvp_heff_contract_noalloc.restype = C.c_int


def heff_contract_noalloc(L, W, R, x, y, stream=None):
    """y = H_eff x (FP64) with no device allocation (scratch in a fixed device array)."""
    ml, mr, wl, wr, d = _check_site_args(L, W, R, x, y)
    Wc, wp = _host(W)
    buf = C.create_string_buffer(512)
    s = _lib.tdvp_heff_contract_noalloc(C.byref(SiteDims(ml, mr, wl, wr, d)), _ptr(L), wp, _ptr(R), _ptr(x),
                                        _ptr(y), _stream(stream), buf, 512)
    if s != 0:
        raise TDVPError(s, buf.value.decode())


_lib.tdvp_checkpoint_write.argtypes = [C.c_char_p, C.c_void_p]
_lib.tdvp_checkpoint_write.restype = C.c_int
_lib.tdvp_checkpoint_read_header.argtypes = [C.c_char_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_void_p,
                                              C.c_int]
_lib.tdvp_checkpoint_read_header.restype = C.c_int
_lib.tdvp_checkpoint_read.argtypes = [C.c_char_p, C.c_int, C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]
_lib.tdvp_checkpoint_read.restype = C.c_int
_lib.tdvp_checkpoint_last_error.argtypes = []
_lib.tdvp_checkpoint_last_error.restype = C.c_char_p
_lib.tdvp_save.argtypes = [_h, C.c_char_p]
_lib.tdvp_save.restype = C.c_int
_lib.tdvp_load.argtypes = [C.c_char_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(_h)]
_lib.tdvp_load.restype = C.c_int


def _ckpt_chk(s):
    if s != 0:
        raise TDVPError(s, _lib.tdvp_checkpoint_last_error().decode())


def write_checkpoint(path, mps):
    """Writes host site tensors (complex128 [m_i, d, m_{i+1}]) to a checkpoint file (host only)."""
    dims = [mps[0].shape[0]] + [a.shape[2] for a in mps]
    pinned = _Pinned(mps, dims)
    _ckpt_chk(_lib.tdvp_checkpoint_write(os.fsencode(path), C.cast(C.pointer(pinned.desc(mps[0].shape[1])),
                                                                  C.c_void_p)))


def checkpoint_header(path):
    n, d = C.c_int(0), C.c_int(0)
    _ckpt_chk(_lib.tdvp_checkpoint_read_header(os.fsencode(path), C.byref(n), C.byref(d), None, 0))
    dims = (C.c_int * (n.value + 1))()
    _ckpt_chk(_lib.tdvp_checkpoint_read_header(os.fsencode(path), C.byref(n), C.byref(d), C.cast(dims, C.c_void_p),
                                               n.value + 1))
    return n.value, d.value, list(dims)


def read_checkpoint(path):
    """The site tensors of a checkpoint file (host only)."""
    n, d, m = checkpoint_header(path)
    arrs = [np.empty((m[i], d, m[i + 1]), dtype=np.complex128) for i in range(n)]
    ptrs = (C.c_void_p * n)(*[a.ctypes.data for a in arrs])
    dims = (C.c_int * (n + 1))(*m)
    _ckpt_chk(_lib.tdvp_checkpoint_read(os.fsencode(path), n, d, C.cast(dims, C.c_void_p), ptrs))
    return arrs


def declared_symbols(header=HEADER):
    """Names of the entry points include/gse_tdvp.h declares."""
    import re
    txt = open(header).read()
    return sorted(set(re.findall(r"TDVP_API\s+[\w\s\*]+?\b(tdvp_\w+)\s*\(", txt)))


def default_options(**kw):
    o = Options()
    _lib.tdvp_default_options(C.byref(o))
    for k, v in kw.items():
        if k == "tau":
            v = complex(v)
            o.tau_re, o.tau_im = v.real, v.imag
        else:
            setattr(o, k, v)
    return o


class _Pinned:
    """Keeps ctypes views of a list of host arrays alive for one call."""

    def __init__(self, arrays, dims):
        self.arrays = [np.ascontiguousarray(a, dtype=np.complex128) for a in arrays]
        self.dims = (C.c_int * len(dims))(*dims)
        self.ptrs = (C.c_void_p * len(self.arrays))(*[a.ctypes.data for a in self.arrays])

    def desc(self, d):
        return _Desc(len(self.arrays), d, self.dims, self.ptrs)


class GseTdvp:
    """One GSE-TDVP1 state on the GPU (wraps a tdvp_handle)."""

    def __init__(self, mps, mpo, stream=None, **opts):
        mps_dims = [mps[0].shape[0]] + [a.shape[2] for a in mps]
        mpo_dims = [mpo[0].shape[0]] + [w.shape[3] for w in mpo]
        d = mps[0].shape[1]
        self._m = _Pinned(mps, mps_dims)
        self._w = _Pinned(mpo, mpo_dims)
        self.n = len(mps)
        self.d = d
        self.opts = default_options(**opts)
        h = _h()
        s = _lib.tdvp_create(C.byref(self._m.desc(d)), C.byref(self._w.desc(d)), C.byref(self.opts),
                             C.c_void_p(stream or 0), C.byref(h))
        if s != 0:
            raise TDVPError(s, "tdvp_create failed")
        self.h = h
        del self._m, self._w

    @classmethod
    def load(cls, path, mpo, stream=None, **opts):
        """A handle created from a checkpoint file (tdvp_load)."""
        self = cls.__new__(cls)
        mpo_dims = [mpo[0].shape[0]] + [w.shape[3] for w in mpo]
        n, d, _ = checkpoint_header(path)
        self.n, self.d = n, d
        self._w = _Pinned(mpo, mpo_dims)
        self.opts = default_options(**opts)
        h = _h()
        st = _lib.tdvp_load(os.fsencode(path), C.byref(self._w.desc(d)), C.byref(self.opts), C.c_void_p(stream or 0),
                            C.byref(h))
        del self._w
        if st != 0:
            raise TDVPError(st, _lib.tdvp_checkpoint_last_error().decode() or "tdvp_load failed")
        self.h = h
        return self

    def save(self, path):
        """Writes the current state to a checkpoint file (tdvp_save)."""
        self._chk(_lib.tdvp_save(self.h, os.fsencode(path)))

    def _chk(self, s):
        if s != 0:
            raise TDVPError(s, _lib.tdvp_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            _lib.tdvp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_options(self, **kw):
        for k, v in kw.items():
            if k == "tau":
                v = complex(v)
                self.opts.tau_re, self.opts.tau_im = v.real, v.imag
            else:
                setattr(self.opts, k, v)
        self._chk(_lib.tdvp_set_options(self.h, C.byref(self.opts)))

    def canonicalize(self, site):
        self._chk(_lib.tdvp_canonicalize(self.h, site))

    def expand_basis(self, k, weights=None):
        w = None
        if weights is not None:
            w = (C.c_double * len(weights))(*weights)
        self._chk(_lib.tdvp_expand_basis(self.h, k, C.cast(w, C.c_void_p) if w is not None else None))

    def apply_krylov(self):
        """State <- normalised, compressed (1 - i tau H)|psi> (one Krylov vector, Eq. 10)."""
        self._chk(_lib.tdvp_apply_krylov(self.h))

    def sweep(self, dt, kind=REAL):
        self._chk(_lib.tdvp_sweep(self.h, dt, kind))

    def step(self, dt, kind, k, weights=None):
        """One GSE-TDVP1 time step: expand (steps 1-2) then sweep (step 3)."""
        self.expand_basis(k, weights)
        self.sweep(dt, kind)

    def krylov_memory(self, max_bytes=-1.0):
        """Sets the device-byte budget of the Krylov step's density environments (0: half the
        free memory; < 0: unchanged) and returns the checkpoint spacing of the last Krylov step."""
        seg = C.c_int(0)
        self._chk(_lib.tdvp_krylov_memory(self.h, float(max_bytes), C.byref(seg)))
        return seg.value

    def krylov_precision(self, precision):
        """Arithmetic of the Krylov vectors' contractions (-1: the handle's precision)."""
        self._chk(_lib.tdvp_set_krylov_precision(self.h, int(precision)))

    def krylov_method(self, method):
        """KRYLOV_DENSITY_MATRIX (default) or KRYLOV_ZIPUP for the Krylov vectors of Eq. 10."""
        self._chk(_lib.tdvp_set_krylov_method(self.h, int(method)))

    def sweep2(self, dt, kind=REAL):
        """One two-site TDVP step (TDVP2), truncating with eps and chi_max in both time kinds."""
        self._chk(_lib.tdvp_sweep2(self.h, dt, kind))

    def _local_vectors(self, n, **ts):
        """x and y of a local operator: contiguous CUDA complex128 tensors of n entries (n None:
        the index is out of range, which the library itself refuses)."""
        for name, t in ts.items():
            if not (t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch.complex128"):
                raise ValueError(f"{name} must be a contiguous CUDA complex128 tensor")
            if n is not None and t.numel() != n:
                raise ValueError(f"{name} has {t.numel()} entries, the local space has {n}")

    def _site_size(self, site):
        if not 0 <= site < self.n:
            return None
        m = self.bond_dims()
        return m[site] * self.d * m[site + 1]

    def heff_apply(self, site, x, y, precision=PREC_FP64):
        self._local_vectors(self._site_size(site), x=x, y=y)
        self._chk(_lib.tdvp_heff_apply(self.h, site, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                       precision))

    def keff_apply(self, bond, x, y, precision=PREC_FP64):
        self._local_vectors(self.bond_dims()[bond] ** 2 if 1 <= bond < self.n else None, x=x, y=y)
        self._chk(_lib.tdvp_keff_apply(self.h, bond, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                       precision))

    def evolve_site(self, site, x, y, delta, kind=REAL, precision=PREC_FP64):
        self._local_vectors(self._site_size(site), x=x, y=y)
        it = C.c_int(0)
        self._chk(_lib.tdvp_evolve_site(self.h, site, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                        delta, kind, precision, C.byref(it)))
        return it.value

    def energy(self):
        v = C.c_double()
        self._chk(_lib.tdvp_energy(self.h, C.byref(v)))
        return v.value

    def norm(self):
        v = C.c_double()
        self._chk(_lib.tdvp_norm(self.h, C.byref(v)))
        return v.value

    def expect_local(self, op, site):
        op = np.ascontiguousarray(op, dtype=np.complex128)
        out = (C.c_double * 2)()
        self._chk(_lib.tdvp_expect_local(self.h, C.c_void_p(op.ctypes.data), site, out))
        return complex(out[0], out[1])

    def expect_mpo(self, mpo):
        """<psi|O|psi>/<psi|psi> for an operator O given as an MPO (list of [wl, d, d, wr])."""
        dims = [mpo[0].shape[0]] + [w.shape[3] for w in mpo]
        pw = _Pinned(mpo, dims)
        out = (C.c_double * 2)()
        self._chk(_lib.tdvp_expect_mpo(self.h, C.byref(pw.desc(self.d)), out))
        return complex(out[0], out[1])

    def bond_dims(self):
        out = (C.c_int * (self.n + 1))()
        self._chk(_lib.tdvp_bond_dims(self.h, out))
        return list(out)

    def bond_charges(self, phys=(1, -1)):
        """U(1) charge of every index of bonds 0..N (lists), read off the state's zero pattern
        from charge 0 at the left end; phys: the d local charges (2 S^z for spin 1/2)."""
        m = self.bond_dims()
        ph = (C.c_int * self.d)(*phys)
        out = (C.c_int * sum(m))()
        self._chk(_lib.tdvp_bond_charges(self.h, ph, out))
        q, o = [], 0
        for mb in m:
            q.append(list(out[o:o + mb]))
            o += mb
        return q

    def bond_sectors(self, bond, phys=(1, -1), max_sectors=4096):
        """([(charge, dim, offset), ...], contiguous) of one bond."""
        ph = (C.c_int * self.d)(*phys)
        q, dm, off = (C.c_int * max_sectors)(), (C.c_int * max_sectors)(), (C.c_int * max_sectors)()
        n, cont = C.c_int(), C.c_int()
        self._chk(_lib.tdvp_bond_sectors(self.h, ph, bond, max_sectors, q, dm, off, C.byref(n), C.byref(cont)))
        if n.value > max_sectors:
            return self.bond_sectors(bond, phys, n.value)
        return [(q[i], dm[i], off[i]) for i in range(n.value)], bool(cont.value)

    def center(self):
        v = C.c_int()
        self._chk(_lib.tdvp_center(self.h, C.byref(v)))
        return v.value

    def trunc_stats(self):
        out = (C.c_double * 13)()
        self._chk(_lib.tdvp_trunc_stats(self.h, out))
        return dict(disc_k=out[0], disc_m=out[1], disc_eps=out[2], added=int(out[3]),
                    lanczos_iters=int(out[4]), lanczos_calls=int(out[5]), svd_calls=int(out[6]),
                    svd_blocked_calls=int(out[7]), svd_blocks=int(out[8]), svd_sweeps=int(out[9]),
                    svd_max_sweeps=int(out[10]), svd_large_blocks=int(out[11]), svd_max_block=int(out[12]))

    def profile(self, enable=True):
        self._chk(_lib.tdvp_profile(self.h, 1 if enable else 0))

    def profile_read(self):
        out = (C.c_double * 3)()
        self._chk(_lib.tdvp_profile_read(self.h, out))
        return dict(applies=int(out[0]), ms=out[1], flops=out[2])

    PHASES = ("lanczos_site", "lanczos_bond", "gauge_sweep", "env", "krylov", "extend", "canonicalize",
              "krylov_right_envs", "krylov_eig", "extend_svd", "svd_prep", "svd_pchol", "svd_jacobi",
              "svd_select", "qr")

    def trace(self, enable=True):
        self._chk(_lib.tdvp_trace(self.h, 1 if enable else 0))

    def trace_read(self):
        out = (C.c_double * len(self.PHASES))()
        self._chk(_lib.tdvp_trace_read(self.h, out, len(self.PHASES)))
        return dict(zip(self.PHASES, list(out)))

    def get_mps(self, alloc=None):
        """The state as host arrays [m_l, d, m_r].  alloc(shape) may supply the destination
        arrays (complex128, C-contiguous; e.g. views of page-locked memory)."""
        m = self.bond_dims()
        shapes = [(m[i], self.d, m[i + 1]) for i in range(self.n)]
        arrs = [np.empty(s, dtype=np.complex128) if alloc is None else alloc(s) for s in shapes]
        for a, s in zip(arrs, shapes):
            if a.shape != s or a.dtype != np.complex128 or not a.flags.c_contiguous:
                raise ValueError("get_mps: destination arrays must be C-contiguous complex128 of the bond shapes")
        ptrs = (C.c_void_p * self.n)(*[a.ctypes.data for a in arrs])
        self._chk(_lib.tdvp_get_mps(self.h, ptrs))
        return arrs


_lib.tdvp_batch_create.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_void_p)]
_lib.tdvp_batch_create.restype = C.c_int
_lib.tdvp_batch_destroy.argtypes = [C.c_void_p]
_lib.tdvp_batch_destroy.restype = C.c_int
_lib.tdvp_batch_handle.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_void_p)]
_lib.tdvp_batch_handle.restype = C.c_int
_lib.tdvp_batch_step.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_double, C.c_int, C.POINTER(C.c_int)]
_lib.tdvp_batch_step.restype = C.c_int
_lib.tdvp_batch_expand_basis.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_int)]
_lib.tdvp_batch_expand_basis.restype = C.c_int
_lib.tdvp_batch_sweep.argtypes = [C.c_void_p, C.c_double, C.c_int, C.POINTER(C.c_int)]
_lib.tdvp_batch_sweep.restype = C.c_int
_lib.tdvp_batch_energy.argtypes = [C.c_void_p, C.POINTER(C.c_double)]
_lib.tdvp_batch_energy.restype = C.c_int
_lib.tdvp_batch_norm.argtypes = [C.c_void_p, C.POINTER(C.c_double)]
_lib.tdvp_batch_norm.restype = C.c_int
_lib.tdvp_batch_last_error.argtypes = [C.c_void_p]
_lib.tdvp_batch_last_error.restype = C.c_char_p


class _Borrowed(GseTdvp):
    """A chain handle owned by a batch (never destroyed through this object)."""

    def close(self):
        self.h = None


class GseTdvpBatch:
    """Independent chains on one GPU, each on its own stream (tdvp_batch_*).

    chains: list of (mps, mpo, options dict).  n_threads <= 0: one host worker per core."""

    def __init__(self, chains, n_threads=0):
        n = len(chains)
        pins, descs_m, descs_w, opts = [], (_Desc * n)(), (_Desc * n)(), (Options * n)()
        self.d = chains[0][0][0].shape[1]
        for i, (mps, mpo, kw) in enumerate(chains):
            pm = _Pinned(mps, [mps[0].shape[0]] + [a.shape[2] for a in mps])
            pw = _Pinned(mpo, [mpo[0].shape[0]] + [w.shape[3] for w in mpo])
            pins += [pm, pw]
            descs_m[i] = pm.desc(mps[0].shape[1])
            descs_w[i] = pw.desc(mps[0].shape[1])
            opts[i] = default_options(**kw)
        b = C.c_void_p()
        s = _lib.tdvp_batch_create(n, C.cast(descs_m, C.c_void_p), C.cast(descs_w, C.c_void_p),
                                   C.cast(opts, C.c_void_p), int(n_threads), C.byref(b))
        if s != 0:
            raise TDVPError(s, "tdvp_batch_create failed")
        self.b = b
        self.n = n
        self.sizes = [len(c[0]) for c in chains]

    def _chk(self, s, status=None):
        if s != 0:
            raise TDVPError(s, _lib.tdvp_batch_last_error(self.b).decode())

    def _status(self):
        return (C.c_int * self.n)()

    def step(self, dt, kind, k, weights=None):
        st = self._status()
        w = None if weights is None else C.cast((C.c_double * len(weights))(*weights), C.c_void_p)
        self._chk(_lib.tdvp_batch_step(self.b, k, w, dt, kind, st))
        return list(st)

    def expand_basis(self, k, weights=None):
        st = self._status()
        w = None if weights is None else C.cast((C.c_double * len(weights))(*weights), C.c_void_p)
        self._chk(_lib.tdvp_batch_expand_basis(self.b, k, w, st))
        return list(st)

    def sweep(self, dt, kind=REAL):
        st = self._status()
        self._chk(_lib.tdvp_batch_sweep(self.b, dt, kind, st))
        return list(st)

    def energies(self):
        out = (C.c_double * self.n)()
        self._chk(_lib.tdvp_batch_energy(self.b, out))
        return list(out)

    def norms(self):
        out = (C.c_double * self.n)()
        self._chk(_lib.tdvp_batch_norm(self.b, out))
        return list(out)

    def chain(self, i):
        """The handle of chain i (owned by the batch; valid while the batch is open)."""
        h = C.c_void_p()
        s = _lib.tdvp_batch_handle(self.b, i, C.byref(h))
        if s != 0:
            raise TDVPError(s, "tdvp_batch_handle")
        c = _Borrowed.__new__(_Borrowed)
        c.h, c.n, c.d = h, self.sizes[i], self.d
        return c

    def close(self):
        if getattr(self, "b", None):
            _lib.tdvp_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
