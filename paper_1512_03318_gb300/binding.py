"""ctypes binding of libmrdmrg with the C names; argument marshalling only.

Device buffers are passed as raw pointers: torch tensors (their data_ptr()) or integers.
Host arrays are numpy arrays converted to the C types of the header."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

MRD_PREC_FP64 = 0
MRD_PREC_TF32 = 1
MRD_PREC_BF16X3 = 2
MRD_PREC_FF = 3
MRD_BASIS_MIXED = 0
MRD_BASIS_REAL = 1
MRD_BASIS_MIXED_REAL = 2
MRD_OPT_GRAPH = 1
MRD_OPT_PER_TASK_LAUNCH = 2
MRD_OPT_AUTOTUNE = 3
MRD_OPT_WAIT_LIMIT_US = 4
MRD_OPT_REAL = 5
MRD_SVD_F32_FF = 0
MRD_SVD_FF = 1
MRD_SVD_F32_F64 = 2
MRD_SVD_F64 = 3
MRD_DMRG_OPT_ENV_FP32 = 1
MRD_DMRG_OPT_REAL = 2
MRD_DMRG_OPT_SVD_PRESWEEPS = 3

_LIB = None
_LIVE = []        # weak references to open handles, closed in creation-reverse order at exit


def _register(obj):
    import weakref
    _LIVE.append(weakref.ref(obj))


def _close_all():
    for r in reversed(_LIVE):
        o = r()
        if o is not None:
            try:
                o.close()
            except Exception:
                pass
    _LIVE.clear()


import atexit  # noqa: E402
atexit.register(_close_all)


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(lib().mrd_launch_count())


def lib_path() -> str:
    return _build.LIB


class MrdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mrdmrg error {code}: {msg}")
        self.code = code


class mrd_model(C.Structure):
    _fields_ = [("lx", C.c_int32), ("ly", C.c_int32), ("flux_p", C.c_int32), ("flux_q", C.c_int32),
                ("t", C.c_double), ("v", C.c_double), ("basis", C.c_int32)]


class mrd_heff_desc(C.Structure):
    _fields_ = [("n_left", C.c_int32), ("left", C.POINTER(C.c_int32)),
                ("n_right", C.c_int32), ("right", C.POINTER(C.c_int32)),
                ("m1", C.c_int32), ("m2", C.c_int32), ("modulus", C.c_int32),
                ("d_l", C.c_int32), ("d_m", C.c_int32), ("d_r", C.c_int32),
                ("c_l", C.POINTER(C.c_int32)), ("c_m", C.POINTER(C.c_int32)), ("c_r", C.POINTER(C.c_int32)),
                ("nnz_i", C.c_int32), ("wi_idx", C.POINTER(C.c_int32)), ("wi_val", C.POINTER(C.c_double)),
                ("nnz_j", C.c_int32), ("wj_idx", C.POINTER(C.c_int32)), ("wj_val", C.POINTER(C.c_double))]


_SIGS = {
    "mrd_version": (C.c_int, []),
    "mrd_launch_count": (C.c_int64, []),
    "mrd_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_void_p]),
    "mrd_destroy": (C.c_int, [C.c_void_p]),
    "mrd_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mrd_release_cached": (C.c_int, [C.c_void_p]),
    "mrd_last_error": (C.c_char_p, [C.c_void_p]),
    "mrd_mpo_build": (C.c_int, [C.c_void_p, C.POINTER(mrd_model), C.POINTER(C.c_void_p)]),
    "mrd_mpo_free": (C.c_int, [C.c_void_p]),
    "mrd_mpo_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "mrd_mpo_bond": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "mrd_mpo_site": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                               C.POINTER(C.c_double)]),
    "mrd_mpo_stats": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_double)]),
    "mrd_heff_create": (C.c_int, [C.c_void_p, C.POINTER(mrd_heff_desc), C.POINTER(C.c_void_p)]),
    "mrd_heff_free": (C.c_int, [C.c_void_p]),
    "mrd_heff_sizes": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "mrd_heff_set_env": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "mrd_heff_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "mrd_heff_flops": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "mrd_heff_table": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "mrd_heff_apply_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "mrd_lanczos": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_double, C.c_int32, C.POINTER(C.c_double),
                              C.POINTER(C.c_int32)]),
    "mrd_heff_rayleigh": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(C.c_double),
                                    C.POINTER(C.c_double)]),
    "mrd_dmrg_create": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_uint64, C.c_int32,
                                  C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_void_p)]),
    "mrd_dmrg_free": (C.c_int, [C.c_void_p]),
    "mrd_two_site_update": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.POINTER(C.c_double),
                                      C.POINTER(C.c_double)]),
    "mrd_sweep": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]),
    "mrd_env_update": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32]),
    "mrd_dmrg_set_option": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64]),
    "mrd_dmrg_memory": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "mrd_dmrg_bond": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "mrd_dmrg_site": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int64),
                                C.POINTER(C.c_double)]),
    "mrd_dmrg_env": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
    "mrd_dmrg_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int32)]),
    "mrd_dmrg_phase_ms": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "mrd_dmrg_set_site": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    "mrd_dmrg_timing": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "mrd_heff_timing": (C.c_int, [C.c_void_p, C.c_int32]),
    "mrd_heff_set_option": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64]),
    "mrd_heff_status": (C.c_int, [C.c_void_p]),
    "mrd_measure_peaks": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "mrd_heff_tc_config": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    "mrd_dmrg_svd_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "mrd_dmrg_svd_trace": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_double),
                                     C.POINTER(C.c_int32)]),
    "mrd_dmrg_schmidt": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                   C.POINTER(C.c_double)]),
    "mrd_heff_timing_collect": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                          C.POINTER(C.c_int32)]),
}


def declared_symbols():
    """Function names declared in include/mrdmrg.h (parsed from the header text)."""
    import re
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "mrdmrg.h")
    with open(hdr) as f:
        text = f.read()
    return sorted(set(re.findall(r"\b(mrd_[a-z0-9_]+)\s*\(", text)))


def lib():
    """Load the shared library (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libmrdmrg not built ({path}); run __graft_entry__.build()")
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def _ptr(x):
    """Raw device pointer of a torch tensor, or an int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32).reshape(-1))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))


def _p32(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _p64f(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class Context:
    def __init__(self, device: int = 0, stream=None):
        h = C.c_void_p()
        rc = lib().mrd_create(C.byref(h), device, _stream_ptr(stream))
        if rc != 0:
            raise MrdError(rc, "mrd_create failed")
        self.h = h
        self.device = device
        _register(self)

    def check(self, rc):
        if rc != 0:
            raise MrdError(rc, lib().mrd_last_error(self.h).decode())

    def release_cached(self):
        """mrd_release_cached: free the device memory the library holds cached for reuse."""
        self.check(lib().mrd_release_cached(self.h))

    def measure_peaks(self):
        """mrd_measure_peaks: (FP32 FMA instr/s, FP64 FMA instr/s, SMs, max SM clock Hz)."""
        out = (C.c_double * 4)()
        self.check(lib().mrd_measure_peaks(self.h, out))
        return tuple(out)

    def set_stream(self, stream):
        self.check(lib().mrd_set_stream(self.h, _stream_ptr(stream)))

    def close(self):
        if self.h:
            lib().mrd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class MPO:
    """Handle of a host-built MPO (mrd_mpo_build). ctx may be None (host only)."""

    def __init__(self, ctx, lx, ly, flux_p, flux_q, t, v, basis=MRD_BASIS_MIXED):
        m = mrd_model(lx, ly, flux_p, flux_q, t, v, basis)
        h = C.c_void_p()
        rc = lib().mrd_mpo_build(ctx.h if ctx is not None else None, C.byref(m), C.byref(h))
        if rc != 0:
            msg = lib().mrd_last_error(ctx.h).decode() if ctx is not None else "mrd_mpo_build failed"
            raise MrdError(rc, msg)
        self.h = h
        _register(self)
        n, mod = C.c_int32(), C.c_int32()
        lib().mrd_mpo_info(h, C.byref(n), C.byref(mod))
        self.n_sites, self.modulus, self.ly = n.value, mod.value, ly

    def bond(self, b):
        d = C.c_int32()
        lib().mrd_mpo_bond(self.h, b, C.byref(d), None)
        ch = np.zeros(2 * d.value, dtype=np.int32)
        lib().mrd_mpo_bond(self.h, b, C.byref(d), _p32(ch))
        return ch.reshape(-1, 2)

    def site(self, j):
        nnz = C.c_int32()
        lib().mrd_mpo_site(self.h, j, C.byref(nnz), None, None)
        idx = np.zeros(4 * nnz.value, dtype=np.int32)
        val = np.zeros(2 * nnz.value, dtype=np.float64)
        lib().mrd_mpo_site(self.h, j, C.byref(nnz), _p32(idx), _p64f(val))
        return idx.reshape(-1, 4), val[0::2] + 1j * val[1::2]

    def stats(self, first, count):
        """(mean bond dimension, largest, mean fill, nonzero entries) of sites first ..
        first+count-1 and the bonds to their left (mrd_mpo_stats)."""
        out = (C.c_double * 4)()
        rc = lib().mrd_mpo_stats(self.h, first, count, out)
        if rc != 0:
            raise MrdError(rc, "mrd_mpo_stats: bad site range")
        return out[0], int(out[1]), out[2], int(out[3])

    def close(self):
        if getattr(self, "h", None):
            lib().mrd_mpo_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class mrd_dmrg_params(C.Structure):
    _fields_ = [("chi", C.c_int32), ("svd_cutoff", C.c_double), ("lanczos_max_iter", C.c_int32),
                ("lanczos_tol", C.c_double), ("prec", C.c_int32), ("refine_iter", C.c_int32),
                ("refine_tol", C.c_double), ("lanczos_restarts", C.c_int32), ("svd_mode", C.c_int32),
                ("refine_prec", C.c_int32)]


class DMRG:
    """Finite two-site DMRG state on the device (mrd_dmrg_*)."""

    def __init__(self, ctx, mpo, n_part, k_tot, chi, seed=1234, center=0, caps=None):
        self.ctx, self.mpo = ctx, mpo
        h = C.c_void_p()
        cp = co = None
        if caps is not None:     # list over bonds of lists of (N, K, dim)
            flat = [x for bond in caps for t in bond for x in t]
            offs = np.cumsum([0] + [len(b) for b in caps]).astype(np.int64)
            self._caps = (np.array(flat, dtype=np.int32), offs)
            cp, co = _p32(self._caps[0]), self._caps[1].ctypes.data_as(C.POINTER(C.c_int64))
        ctx.check(lib().mrd_dmrg_create(ctx.h, mpo.h, n_part, k_tot, chi, seed, center, cp, co, C.byref(h)))
        self.h = h
        _register(self)

    @staticmethod
    def params(chi, cutoff=1e-14, max_iter=30, tol=1e-13, prec=MRD_PREC_FP64, refine_iter=0, refine_tol=1e-13,
               restarts=0, svd_mode=None, refine_prec=None):
        # FP64 updates stay in FP64 throughout; reduced-precision ones use FP32 pre-sweeps and
        # float-float sweeps for the SVD, and float-float for the refinement, the environment
        # updates and the SVD's GEMMs
        if svd_mode is None:
            svd_mode = MRD_SVD_F64 if prec == MRD_PREC_FP64 else MRD_SVD_F32_FF
        if refine_prec is None:
            refine_prec = MRD_PREC_FP64 if prec == MRD_PREC_FP64 else MRD_PREC_FF
        return mrd_dmrg_params(chi, cutoff, max_iter, tol, prec, refine_iter, refine_tol, restarts, svd_mode,
                               refine_prec)

    def update(self, i, direction, params):
        e, t = C.c_double(), C.c_double()
        self.ctx.check(lib().mrd_two_site_update(self.h, i, direction, C.byref(params), C.byref(e), C.byref(t)))
        return e.value, t.value

    def sweep(self, params):
        e = C.c_double()
        self.ctx.check(lib().mrd_sweep(self.h, C.byref(params), C.byref(e)))
        return e.value

    def set_option(self, option, value):
        """mrd_dmrg_set_option (MRD_DMRG_OPT_ENV_FP32, MRD_DMRG_OPT_REAL, MRD_DMRG_OPT_SVD_PRESWEEPS)."""
        self.ctx.check(lib().mrd_dmrg_set_option(self.h, option, int(value)))

    def memory(self):
        """(environment bytes, environments built, MPS bytes, complex64 storage) of the state."""
        out = (C.c_int64 * 4)()
        self.ctx.check(lib().mrd_dmrg_memory(self.h, out))
        return tuple(out)

    def env_update(self, site, direction, prec=MRD_PREC_FP64):
        """mrd_env_update: rebuild the left environment of bond site+1 (direction +1) or the right
        environment of bond site (direction -1) from the neighbouring one."""
        self.ctx.check(lib().mrd_env_update(self.h, site, direction, prec))

    def bond(self, b):
        n = C.c_int32()
        lib().mrd_dmrg_bond(self.h, b, C.byref(n), None)
        out = np.zeros(3 * max(n.value, 1), dtype=np.int32)
        lib().mrd_dmrg_bond(self.h, b, C.byref(n), _p32(out))
        return out[: 3 * n.value].reshape(-1, 3)

    def site(self, j):
        mode, ln = C.c_int32(), C.c_int64()
        self.ctx.check(lib().mrd_dmrg_site(self.h, j, C.byref(mode), C.byref(ln), None))
        buf = np.zeros(2 * max(ln.value, 1), dtype=np.float64)
        self.ctx.check(lib().mrd_dmrg_site(self.h, j, C.byref(mode), C.byref(ln), _p64f(buf)))
        return mode.value, (buf[0::2] + 1j * buf[1::2])[: ln.value]

    def env(self, b, side):
        ln = C.c_int64()
        self.ctx.check(lib().mrd_dmrg_env(self.h, b, side, C.byref(ln), None))
        if ln.value < 0:
            return None
        buf = np.zeros(2 * max(ln.value, 1), dtype=np.float64)
        self.ctx.check(lib().mrd_dmrg_env(self.h, b, side, C.byref(ln), _p64f(buf)))
        return (buf[0::2] + 1j * buf[1::2])[: ln.value]

    def env_len(self, b, side):
        """Length (complex elements) of the environment at bond b (side 0 left, 1 right); -1 if not built."""
        ln = C.c_int64()
        self.ctx.check(lib().mrd_dmrg_env(self.h, b, side, C.byref(ln), None))
        return ln.value

    def set_site(self, j, host_ptr):
        """host_ptr: address of complex128 data (e.g. a pinned torch tensor's data_ptr())."""
        self.ctx.check(lib().mrd_dmrg_set_site(self.h, j, _ptr(host_ptr)))

    def site_into(self, j, host_tensor):
        """Copy MPS tensor j into a host tensor (complex128, numel >= len)."""
        mode, ln = C.c_int32(), C.c_int64()
        self.ctx.check(lib().mrd_dmrg_site(self.h, j, C.byref(mode), C.byref(ln), None))
        if host_tensor.numel() < ln.value:
            raise ValueError(f"site {j} has {ln.value} elements; the host tensor holds {host_tensor.numel()}")
        self.ctx.check(lib().mrd_dmrg_site(self.h, j, C.byref(mode), C.byref(ln),
                                           C.cast(C.c_void_p(host_tensor.data_ptr()), C.POINTER(C.c_double))))
        return ln.value

    def site_len(self, j):
        mode, ln = C.c_int32(), C.c_int64()
        self.ctx.check(lib().mrd_dmrg_site(self.h, j, C.byref(mode), C.byref(ln), None))
        return ln.value

    def timing(self, on=True):
        ms = (C.c_double * 4)()
        n = (C.c_int64 * 2)()
        self.ctx.check(lib().mrd_dmrg_timing(self.h, 1 if on else 0, ms, n))
        return list(ms), list(n)

    def phase_ms(self):
        """[tables, theta, lanczos, svd, tensors, env] ms of the last update."""
        f = (C.c_double * 8)()
        self.ctx.check(lib().mrd_dmrg_phase_ms(self.h, f))
        return list(f)[:6]

    def svd_sweeps(self):
        f = (C.c_double * 8)()
        self.ctx.check(lib().mrd_dmrg_phase_ms(self.h, f))
        return int(f[6]), int(f[7])

    def schmidt(self):
        """(bond, {(N, K): Schmidt values}) of the bond cut by the last update (mrd_dmrg_schmidt)."""
        b, n = C.c_int32(), C.c_int64()
        self.ctx.check(lib().mrd_dmrg_schmidt(self.h, C.byref(b), C.byref(n), None, None))
        nk = np.zeros(2 * max(n.value, 1), dtype=np.int32)
        val = np.zeros(max(n.value, 1), dtype=np.float64)
        self.ctx.check(lib().mrd_dmrg_schmidt(self.h, C.byref(b), C.byref(n), _p32(nk),
                                              val.ctypes.data_as(C.POINTER(C.c_double))))
        out = {}
        for j in range(n.value):
            out.setdefault((int(nk[2 * j]), int(nk[2 * j + 1])), []).append(val[j])
        return b.value, {k: np.sort(np.array(v))[::-1] for k, v in out.items()}

    def svd_stats(self):
        """(sweep ms, element-pairs tested, element-pairs rotated, sweeps, FP32 pre-sweep ms, svd_mode,
        columns entering the final sweeps, columns of all blocks)."""
        f = (C.c_double * 8)()
        self.ctx.check(lib().mrd_dmrg_svd_stats(self.h, f))
        return tuple(f)

    def svd_trace(self, cap=256, times=False):
        """Column pairs rotated per Jacobi sweep of the last block SVD: (FP32 pre-sweeps, final);
        with times=True also the host ms of each sweep, in the same two lists."""
        out, ms, n2 = (C.c_int32 * cap)(), (C.c_double * cap)(), (C.c_int32 * 2)()
        self.ctx.check(lib().mrd_dmrg_svd_trace(self.h, cap, out, ms, n2))
        k = min(cap, n2[0] + n2[1])
        v, t = list(out)[:k], list(ms)[:k]
        if times:
            return v[:n2[0]], v[n2[0]:], t[:n2[0]], t[n2[0]:]
        return v[:n2[0]], v[n2[0]:]

    def stats(self):
        e, t, it = C.c_double(), C.c_double(), C.c_int32()
        lib().mrd_dmrg_stats(self.h, C.byref(e), C.byref(t), C.byref(it))
        return e.value, t.value, it.value

    def close(self):
        if getattr(self, "h", None):
            lib().mrd_dmrg_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Heff:
    """Two-site H_eff problem (mrd_heff_create / set_env / apply)."""

    def __init__(self, ctx: Context, left, right, m1, m2, modulus, cl, cm, cr, wi_idx, wi_val, wj_idx, wj_val):
        self.ctx = ctx
        keep = {}
        keep["left"] = _i32(left)
        keep["right"] = _i32(right)
        keep["cl"], keep["cm"], keep["cr"] = _i32(cl), _i32(cm), _i32(cr)
        keep["wi_idx"], keep["wj_idx"] = _i32(wi_idx), _i32(wj_idx)
        wv = np.asarray(wi_val, dtype=np.complex128).reshape(-1)
        keep["wi_val"] = _f64(np.stack([wv.real, wv.imag], axis=1))
        wv = np.asarray(wj_val, dtype=np.complex128).reshape(-1)
        keep["wj_val"] = _f64(np.stack([wv.real, wv.imag], axis=1))
        d = mrd_heff_desc()
        d.n_left, d.left = len(keep["left"]) // 3, _p32(keep["left"])
        d.n_right, d.right = len(keep["right"]) // 3, _p32(keep["right"])
        d.m1, d.m2, d.modulus = m1, m2, modulus
        d.d_l, d.d_m, d.d_r = len(keep["cl"]) // 2, len(keep["cm"]) // 2, len(keep["cr"]) // 2
        d.c_l, d.c_m, d.c_r = _p32(keep["cl"]), _p32(keep["cm"]), _p32(keep["cr"])
        d.nnz_i, d.wi_idx, d.wi_val = len(keep["wi_idx"]) // 4, _p32(keep["wi_idx"]), _p64f(keep["wi_val"])
        d.nnz_j, d.wj_idx, d.wj_val = len(keep["wj_idx"]) // 4, _p32(keep["wj_idx"]), _p64f(keep["wj_val"])
        h = C.c_void_p()
        ctx.check(lib().mrd_heff_create(ctx.h, C.byref(d), C.byref(h)))
        self.h = h
        _register(self)
        t, l, r = C.c_int64(), C.c_int64(), C.c_int64()
        lib().mrd_heff_sizes(h, C.byref(t), C.byref(l), C.byref(r))
        self.theta_len, self.lenv_len, self.renv_len = t.value, l.value, r.value

    def set_env(self, lenv, renv):
        self.ctx.check(lib().mrd_heff_set_env(self.h, _ptr(lenv), _ptr(renv)))

    def set_option(self, option, value):
        """mrd_heff_set_option (MRD_OPT_GRAPH, MRD_OPT_PER_TASK_LAUNCH, MRD_OPT_AUTOTUNE,
        MRD_OPT_WAIT_LIMIT_US)."""
        self.ctx.check(lib().mrd_heff_set_option(self.h, option, int(value)))

    def status(self):
        """mrd_heff_status: raises MrdError (MRD_E_TIMEOUT) if a tensor-core wait gave up."""
        self.ctx.check(lib().mrd_heff_status(self.h))

    def tc_config(self):
        """(columns per tile, stages, task order, source) of the tensor-core GEMM (mrd_heff_tc_config)."""
        c = (C.c_int32 * 4)()
        self.ctx.check(lib().mrd_heff_tc_config(self.h, c))
        return tuple(c)

    def apply(self, theta_in, theta_out, prec=MRD_PREC_FP64):
        self.ctx.check(lib().mrd_heff_apply(self.h, _ptr(theta_in), _ptr(theta_out), prec))

    def lanczos(self, theta, max_iter=30, tol=1e-13, prec=MRD_PREC_FP64):
        """In place: theta (device) -> ground vector; returns (energy, matvecs)."""
        e, it = C.c_double(), C.c_int32()
        self.ctx.check(lib().mrd_lanczos(self.h, _ptr(theta), max_iter, tol, prec, C.byref(e), C.byref(it)))
        return e.value, it.value

    def rayleigh(self, theta, prec=MRD_PREC_FP64):
        e, r = C.c_double(), C.c_double()
        self.ctx.check(lib().mrd_heff_rayleigh(self.h, _ptr(theta), prec, C.byref(e), C.byref(r)))
        return e.value, r.value

    def apply_noalloc(self, theta_in, theta_out):
        """mrd_heff_apply_noalloc: same product, no device allocation (static scratch)."""
        self.ctx.check(lib().mrd_heff_apply_noalloc(self.h, _ptr(theta_in), _ptr(theta_out)))

    def flops(self):
        """(definition-order, executed, executed step 1, executed step 2) real flops."""
        f = (C.c_double * 4)()
        self.ctx.check(lib().mrd_heff_flops(self.h, f))
        return f[0], f[1], f[2], f[3]

    def timing(self, on=True):
        self.ctx.check(lib().mrd_heff_timing(self.h, 1 if on else 0))

    def timing_collect(self):
        a, b, n = C.c_double(), C.c_double(), C.c_int32()
        self.ctx.check(lib().mrd_heff_timing_collect(self.h, C.byref(a), C.byref(b), C.byref(n)))
        return a.value, b.value, n.value

    def table(self, which):
        n = C.c_int64()
        self.ctx.check(lib().mrd_heff_table(self.h, which, None, C.byref(n)))
        width = 8 if which == 0 else 6
        rows = np.zeros(max(1, n.value) * width, dtype=np.int64)
        self.ctx.check(lib().mrd_heff_table(self.h, which, rows.ctypes.data_as(C.POINTER(C.c_int64)), C.byref(n)))
        return rows[: n.value * width].reshape(-1, width)

    def close(self):
        if getattr(self, "h", None):
            lib().mrd_heff_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
