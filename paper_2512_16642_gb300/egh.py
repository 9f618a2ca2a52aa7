"""Thin ctypes binding of the egh C ABI (include/egh.h).

Argument marshalling only: every numerical step runs in the CUDA kernels of
libegh.so.  Buffers may be torch tensors (CUDA tensors are passed as device
pointers on the current torch stream; CPU tensors as host pointers) or numpy
arrays (host pointers).  Loading fails loudly when the library is missing;
there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libegh.so")

EGH_OK, EGH_EINVAL, EGH_ENOMEM, EGH_ECUDA, EGH_ENOTPD, EGH_ESTATE, EGH_ETIMEOUT = range(7)
EGH_MU_ABS, EGH_MU_REL_MEANDIAG, EGH_MU_REL_MAXEIG = range(3)
EGH_PREC_FP32, EGH_PREC_MIXED, EGH_PREC_MIXED_FP64 = range(3)

_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)


class egh_config(ctypes.Structure):
    _fields_ = [
        ("nz", ctypes.c_int32), ("nx", ctypes.c_int32),
        ("dz", ctypes.c_double), ("dx", ctypes.c_double),
        ("nsponge", ctypes.c_int32), ("sponge_R", ctypes.c_double),
        ("dt", ctypes.c_double), ("nt", ctypes.c_int32),
        ("nrec", ctypes.c_int32), ("rec_iz", _i32p), ("rec_ix", _i32p),
        ("nfreq", ctypes.c_int32), ("freq_hz", _f64p),
        ("batch_receivers", ctypes.c_int32), ("dft_chunk", ctypes.c_int32),
        ("gram_splits", ctypes.c_int32), ("fd_rows", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("fd_kernel", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 2),
    ]


class egh_stats(ctypes.Structure):
    _fields_ = [
        ("green_ms", ctypes.c_double), ("hessian_ms", ctypes.c_double),
        ("factor_ms", ctypes.c_double), ("deblur_ms", ctypes.c_double),
        ("pde_solves", ctypes.c_int64), ("point_steps", ctypes.c_int64),
        ("deblur_sources", ctypes.c_int64), ("mu", ctypes.c_double),
        ("nz_pad", ctypes.c_int32), ("nx_pad", ctypes.c_int32), ("pitch", ctypes.c_int32),
        ("batch_receivers", ctypes.c_int32), ("dft_chunk", ctypes.c_int32),
        ("gram_splits", ctypes.c_int32), ("kernel_launches", ctypes.c_int64),
        ("fd_rows", ctypes.c_int32), ("pad_", ctypes.c_int32),
        ("fd_ms", ctypes.c_double), ("dft_ms", ctypes.c_double),
        ("fd_launches", ctypes.c_int64), ("dft_launches", ctypes.c_int64),
        ("gram_ms", ctypes.c_double), ("fd_steps", ctypes.c_int64),
        ("fd_kernel", ctypes.c_int32), ("fd_tiles", ctypes.c_int32),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class egh_server_config(ctypes.Structure):
    _fields_ = [
        ("hbm_budget_bytes", ctypes.c_int64), ("slots", ctypes.c_int32),
        ("max_batch_sources", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 3),
    ]


class egh_server_stats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("rejected", ctypes.c_int64),
        ("sources_done", ctypes.c_int64), ("batches", ctypes.c_int64),
        ("peak_bytes_in_use", ctypes.c_int64), ("peak_in_flight", ctypes.c_int32),
        ("pad_", ctypes.c_int32), ("p50_s", ctypes.c_double), ("p99_s", ctypes.c_double),
        ("mean_s", ctypes.c_double), ("span_s", ctypes.c_double),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "pad_"}


_vp = ctypes.c_void_p
_SIGS = {
    "egh_create": ([ctypes.POINTER(egh_config), ctypes.POINTER(_vp)], ctypes.c_int),
    "egh_destroy": ([_vp], None),
    "egh_green": ([_vp, _vp, _vp], ctypes.c_int),
    "egh_deblur_diag": ([_vp, _vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp], ctypes.c_int),
    "egh_sample_receivers": ([ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint64, _vp],
                             ctypes.c_int),
    "egh_green_bandlimited": ([_vp, _vp, _vp, ctypes.c_int32, ctypes.c_int32, _vp], ctypes.c_int),
    "egh_hessian": ([_vp, ctypes.c_int, ctypes.c_double, _f64p, _vp], ctypes.c_int),
    "egh_factor": ([_vp, _i32p, _vp], ctypes.c_int),
    "egh_deblur": ([_vp, _vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp], ctypes.c_int),
    "egh_deblur_freq": ([_vp, _vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp], ctypes.c_int),
    "egh_forward": ([_vp, _vp, ctypes.c_int32, _i32p, _i32p, _vp, _vp, _vp], ctypes.c_int),
    "egh_get_green": ([_vp, ctypes.c_int32, ctypes.c_int32, _vp], ctypes.c_int),
    "egh_get_hessian": ([_vp, ctypes.c_int32, _vp], ctypes.c_int),
    "egh_get_stats": ([_vp, ctypes.POINTER(egh_stats)], ctypes.c_int),
    "egh_gram_noalloc": ([_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _vp, _vp], ctypes.c_int),
    "egh_last_error": ([_vp], ctypes.c_char_p),
    "egh_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "egh_version": ([], ctypes.c_int32),
    "egh_release_green": ([_vp], ctypes.c_int),
    "egh_test_expire_wait": ([_vp, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
    "egh_set_refinement": ([_vp, ctypes.c_double], ctypes.c_int),
    "egh_export_green": ([_vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp], ctypes.c_int),
    "egh_import_green": ([_vp, _vp, _vp], ctypes.c_int),
    "egh_diag_sum": ([_vp, _f64p], ctypes.c_int),
    "egh_set_mu": ([_vp, ctypes.c_double, _vp], ctypes.c_int),
    "egh_save": ([_vp, ctypes.c_char_p], ctypes.c_int),
    "egh_load": ([_vp, ctypes.c_char_p], ctypes.c_int),
    "egh_set_synthesis_frequencies": ([_vp, _f64p, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
    "egh_get_refinement": ([_vp, _f64p, _i32p], ctypes.c_int),
    "egh_server_test_expire_wait": ([_vp, ctypes.c_int32], ctypes.c_int),
    "egh_batch_create": ([ctypes.POINTER(_vp), ctypes.c_int32, ctypes.POINTER(_vp)], ctypes.c_int),
    "egh_batch_factor": ([_vp, _i32p, _i32p, _vp], ctypes.c_int),
    "egh_batch_last_error": ([_vp], ctypes.c_char_p),
    "egh_batch_destroy": ([_vp], None),
    "egh_server_create": ([ctypes.POINTER(egh_server_config), ctypes.POINTER(_vp)], ctypes.c_int),
    "egh_server_add_set": ([_vp, ctypes.c_int32, ctypes.c_int32, _f64p, ctypes.c_double, ctypes.c_int32,
                            ctypes.c_int32, _vp, _i32p], ctypes.c_int),
    "egh_server_submit": ([_vp, ctypes.c_int32, _vp, ctypes.c_int32, ctypes.c_int32, _vp,
                           ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "egh_server_wait": ([_vp, ctypes.c_int64, ctypes.c_double, _f64p], ctypes.c_int),
    "egh_server_drain": ([_vp, ctypes.c_double], ctypes.c_int),
    "egh_server_get_stats": ([_vp, ctypes.POINTER(egh_server_stats)], ctypes.c_int),
    "egh_server_reset_stats": ([_vp], ctypes.c_int),
    "egh_server_hold": ([_vp, ctypes.c_int32], ctypes.c_int),
    "egh_server_last_error": ([_vp], ctypes.c_char_p),
    "egh_server_destroy": ([_vp], None),
}
EXPORTS = tuple(_SIGS)

_lib = None


def load(path: str = LIB_PATH):
    """Loads libegh.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"libegh.so not built ({path}); run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        for name, (args, res) in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


class EghError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{status_string(status)}: {msg}")
        self.status = status


def status_string(s):
    return load().egh_status_string(s).decode()


def _check(rc, ctx):
    if rc != EGH_OK:
        raise EghError(rc, load().egh_last_error(ctx).decode())


def _ptr(buf):
    """(pointer, is_cuda_tensor) of a torch tensor or numpy array (must be contiguous)."""
    if isinstance(buf, np.ndarray):
        if not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return buf.ctypes.data, False
    if hasattr(buf, "data_ptr"):
        if not buf.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return buf.data_ptr(), buf.is_cuda
    raise TypeError(f"unsupported buffer type {type(buf)}")


def _stream(stream, any_cuda):
    if stream is not None:
        return int(stream)
    if any_cuda:
        import torch

        return torch.cuda.current_stream().cuda_stream
    return 0


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_i32p)


# ---- the ABI calls, same names -----------------------------------------------------------
def egh_create(nz, nx, dz, dx, nsponge, sponge_R, dt, nt, rec_iz, rec_ix, freq_hz,
               batch_receivers=0, dft_chunk=0, gram_splits=0, fd_rows=0, precision=0, fd_kernel=0):
    lib = load()
    riz, riz_p = _i32(rec_iz)
    rix, rix_p = _i32(rec_ix)
    f = np.ascontiguousarray(freq_hz, dtype=np.float64)
    cfg = egh_config(int(nz), int(nx), float(dz), float(dx), int(nsponge), float(sponge_R), float(dt),
                     int(nt), int(riz.size), riz_p, rix_p, int(f.size), f.ctypes.data_as(_f64p),
                     int(batch_receivers), int(dft_chunk), int(gram_splits), int(fd_rows),
                     int(precision), int(fd_kernel))
    h = _vp()
    _check(lib.egh_create(ctypes.byref(cfg), ctypes.byref(h)), None)
    return h


def egh_destroy(ctx):
    load().egh_destroy(ctx)


def egh_green(ctx, vel, stream=None):
    p, cu = _ptr(vel)
    _check(load().egh_green(ctx, p, _stream(stream, cu)), ctx)


def egh_green_bandlimited(ctx, vel, wavelet, decim, stream=None):
    p, cu = _ptr(vel)
    w = np.ascontiguousarray(wavelet, dtype=np.float32)
    _check(load().egh_green_bandlimited(ctx, p, w.ctypes.data, int(w.size), int(decim),
                                        _stream(stream, cu)), ctx)


def egh_hessian(ctx, mode=EGH_MU_REL_MEANDIAG, mu_param=1e-2, stream=None):
    mu = ctypes.c_double(0.0)
    _check(load().egh_hessian(ctx, int(mode), float(mu_param), ctypes.byref(mu), _stream(stream, True)),
           ctx)
    return mu.value


def egh_factor(ctx, stream=None):
    bad = ctypes.c_int32(-1)
    rc = load().egh_factor(ctx, ctypes.byref(bad), _stream(stream, True))
    if rc == EGH_ENOTPD:
        err = EghError(rc, load().egh_last_error(ctx).decode())
        err.bad_freq = bad.value
        raise err
    _check(rc, ctx)
    return bad.value


def egh_deblur(ctx, resid, ns, nt_d, mult, stream=None):
    pi, ci = _ptr(resid)
    po, co = _ptr(mult)
    _check(load().egh_deblur(ctx, pi, int(ns), int(nt_d), po, _stream(stream, ci or co)), ctx)


def egh_deblur_diag(ctx, resid, ns, nt_d, mult, stream=None):
    pi, ci = _ptr(resid)
    po, co = _ptr(mult)
    _check(load().egh_deblur_diag(ctx, pi, int(ns), int(nt_d), po, _stream(stream, ci or co)), ctx)


def sample_receivers(nrec, nsub, seed, iteration=0):
    """One receiver index drawn from each of nsub contiguous subsets of 0 .. nrec-1 (int32)."""
    out = np.empty(int(nsub), dtype=np.int32)
    _check(load().egh_sample_receivers(int(nrec), int(nsub), int(seed) & (2**64 - 1),
                                       int(iteration) & (2**64 - 1), out.ctypes.data), None)
    return out


def egh_deblur_freq(ctx, resid, ns, nt_d, X, stream=None):
    pi, ci = _ptr(resid)
    px, cx = _ptr(X)
    _check(load().egh_deblur_freq(ctx, pi, int(ns), int(nt_d), px, _stream(stream, ci or cx)), ctx)


def egh_forward(ctx, vel, src_iz, src_ix, wavelet, data, stream=None):
    pv, cv = _ptr(vel)
    siz, siz_p = _i32(src_iz)
    six, six_p = _i32(src_ix)
    w = np.ascontiguousarray(wavelet, dtype=np.float32)
    pd, cd = _ptr(data)
    _check(load().egh_forward(ctx, pv, int(siz.size), siz_p, six_p, w.ctypes.data, pd,
                              _stream(stream, cv or cd)), ctx)


def egh_get_green(ctx, r0, nr, out):
    p, _ = _ptr(out)
    _check(load().egh_get_green(ctx, int(r0), int(nr), p), ctx)


def egh_get_hessian(ctx, factored, out):
    p, _ = _ptr(out)
    _check(load().egh_get_hessian(ctx, int(factored), p), ctx)


def egh_get_stats(ctx):
    st = egh_stats()
    _check(load().egh_get_stats(ctx, ctypes.byref(st)), ctx)
    return st.as_dict()


EXPIRE_GREEN_TRANSFORM, EXPIRE_FD_RESIDENT, EXPIRE_DEBLUR_TRANSFORM = range(3)


def egh_export_green(ctx, k0, nk, out, stream=None):
    p, cu = _ptr(out)
    _check(load().egh_export_green(ctx, int(k0), int(nk), p, _stream(stream, cu)), ctx)


def egh_import_green(ctx, gh, stream=None):
    p, cu = _ptr(gh)
    _check(load().egh_import_green(ctx, p, _stream(stream, cu)), ctx)


def egh_diag_sum(ctx):
    out = ctypes.c_double(0.0)
    _check(load().egh_diag_sum(ctx, ctypes.byref(out)), ctx)
    return out.value


def egh_set_mu(ctx, mu, stream=None):
    _check(load().egh_set_mu(ctx, float(mu), _stream(stream, True)), ctx)


def egh_set_synthesis_frequencies(ctx, all_freq_hz, k0):
    f = np.ascontiguousarray(all_freq_hz, dtype=np.float64)
    _check(load().egh_set_synthesis_frequencies(ctx, f.ctypes.data_as(_f64p), int(f.size), int(k0)), ctx)


def egh_set_refinement(ctx, threshold):
    _check(load().egh_set_refinement(ctx, float(threshold)), ctx)


def egh_get_refinement(ctx, nfreq):
    """(condition bounds [nfreq] float64, refined [nfreq] bool) of the last factorisation."""
    cb = np.zeros(int(nfreq), np.float64)
    rf = np.zeros(int(nfreq), np.int32)
    _check(load().egh_get_refinement(ctx, cb.ctypes.data_as(_f64p), rf.ctypes.data_as(_i32p)), ctx)
    return cb, rf.astype(bool)


def egh_test_expire_wait(ctx, kind, count=1):
    _check(load().egh_test_expire_wait(ctx, int(kind), int(count)), ctx)


def _nbytes(buf):
    if isinstance(buf, np.ndarray):
        return buf.nbytes
    return buf.numel() * buf.element_size()


def egh_gram_noalloc(gh, nrec, nfreq, npts, H, stream=None):
    """Gram of caller-owned device transforms into caller-owned H, allocating nothing."""
    need_gh = 4 * int(nrec) * int(nfreq) * 2 * int(npts)
    need_h = 8 * int(nfreq) * int(nrec) * int(nrec)
    if int(nrec) > 0 and int(nfreq) > 0 and int(npts) > 0:
        if _nbytes(gh) < need_gh:
            raise ValueError(f"gh holds {_nbytes(gh)} bytes, needs {need_gh} (nrec x nfreq x 2 x npts float32)")
        if _nbytes(H) < need_h:
            raise ValueError(f"H holds {_nbytes(H)} bytes, needs {need_h} (nfreq x nrec x nrec complex64)")
    pg, cg = _ptr(gh)
    ph, chh = _ptr(H)
    _check(load().egh_gram_noalloc(pg, int(nrec), int(nfreq), int(npts), ph, _stream(stream, cg or chh)),
           None)


def egh_version():
    return load().egh_version()


# ---- convenience wrapper -------------------------------------------------------------------
class Context:
    """Owns one egh context; methods mirror the ABI and return numpy results where a copy is
    implied (get_green, get_hessian)."""

    def __init__(self, nz, nx, dz, dx, nsponge, sponge_R, dt, nt, rec_iz, rec_ix, freq_hz, **kw):
        self.nz, self.nx, self.ns, self.nt = int(nz), int(nx), int(nsponge), int(nt)
        self.nrec = int(np.size(rec_iz))
        self.freqs = np.asarray(freq_hz, dtype=np.float64)
        self.nf = self.freqs.size
        self.h = egh_create(nz, nx, dz, dx, nsponge, sponge_R, dt, nt, rec_iz, rec_ix, freq_hz, **kw)

    def close(self):
        if self.h:
            egh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def green(self, vel, stream=None):
        egh_green(self.h, vel, stream)

    def green_bandlimited(self, vel, wavelet, decim, stream=None):
        egh_green_bandlimited(self.h, vel, wavelet, decim, stream)

    def hessian(self, mode=EGH_MU_REL_MEANDIAG, mu_param=1e-2, stream=None):
        return egh_hessian(self.h, mode, mu_param, stream)

    def factor(self, stream=None):
        return egh_factor(self.h, stream)

    def deblur(self, resid, mult, stream=None):
        ns, nr, ntd = resid.shape
        egh_deblur(self.h, resid, ns, ntd, mult, stream)
        return mult

    def deblur_diag(self, resid, mult, stream=None):
        ns, nr, ntd = resid.shape
        egh_deblur_diag(self.h, resid, ns, ntd, mult, stream)
        return mult

    def deblur_freq(self, resid, X, stream=None):
        ns, nr, ntd = resid.shape
        egh_deblur_freq(self.h, resid, ns, ntd, X, stream)
        return X

    def forward(self, vel, src_iz, src_ix, wavelet, data, stream=None):
        egh_forward(self.h, vel, src_iz, src_ix, wavelet, data, stream)
        return data

    def get_green(self, r0=0, nr=None):
        nr = self.nrec - r0 if nr is None else nr
        NZ, NX = self.nz + 2 * self.ns, self.nx + 2 * self.ns
        out = np.zeros((nr, self.nf, NZ, NX), dtype=np.complex64)
        egh_get_green(self.h, r0, nr, out)
        return out

    def test_expire_wait(self, kind, count=1):
        egh_test_expire_wait(self.h, kind, count)

    def export_green(self, k0, nk, out, stream=None):
        egh_export_green(self.h, k0, nk, out, stream)

    def import_green(self, gh, stream=None):
        egh_import_green(self.h, gh, stream)

    def diag_sum(self):
        return egh_diag_sum(self.h)

    def set_mu(self, mu, stream=None):
        egh_set_mu(self.h, mu, stream)

    def save(self, path):
        """Writes the factored Hessian set to a file (egh_save)."""
        _check(load().egh_save(self.h, os.fsencode(path)), self.h)

    def load(self, path):
        """Reads a Hessian set written by save into this context and factors it (egh_load)."""
        _check(load().egh_load(self.h, os.fsencode(path)), self.h)

    def set_synthesis_frequencies(self, all_freq_hz, k0):
        egh_set_synthesis_frequencies(self.h, all_freq_hz, k0)

    def transform_buffer(self, nr, nk):
        """Zeroed device buffer [nr][nk][re/im][G] float32 for egh_export_green / egh_import_green."""
        import torch

        st = self.stats()
        G = (st["nz_pad"] * st["pitch"] + 255) // 256 * 256
        return torch.zeros((int(nr), int(nk), 2, G), dtype=torch.float32, device="cuda")

    def set_refinement(self, threshold):
        egh_set_refinement(self.h, threshold)

    def get_refinement(self):
        return egh_get_refinement(self.h, self.nf)

    def release_green(self):
        _check(load().egh_release_green(self.h), self.h)

    def get_hessian(self, factored=False):
        out = np.zeros((self.nf, self.nrec, self.nrec), dtype=np.complex64)
        egh_get_hessian(self.h, 1 if factored else 0, out)
        return out

    def stats(self):
        return egh_get_stats(self.h)


# ---- batched factorisation -------------------------------------------------------------------
class Batch:
    """Contexts (survey patches) factored together in one persistent launch replayed as a CUDA
    graph (egh_batch_* in include/egh.h).  The contexts must outlive the batch."""

    def __init__(self, contexts):
        self._ctxs = list(contexts)
        arr = (_vp * len(self._ctxs))(*[c.h for c in self._ctxs])
        h = _vp()
        rc = load().egh_batch_create(arr, len(self._ctxs), ctypes.byref(h))
        if rc != EGH_OK:
            raise EghError(rc, load().egh_batch_last_error(None).decode())
        self.h = h

    def factor(self, stream=None):
        bc, bf = ctypes.c_int32(-1), ctypes.c_int32(-1)
        rc = load().egh_batch_factor(self.h, ctypes.byref(bc), ctypes.byref(bf), _stream(stream, True))
        if rc != EGH_OK:
            err = EghError(rc, load().egh_batch_last_error(self.h).decode())
            err.bad_ctx, err.bad_freq = bc.value, bf.value
            raise err

    def close(self):
        if self.h:
            load().egh_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- serving ------------------------------------------------------------------------------
def _check_server(rc, sv):
    if rc != EGH_OK:
        raise EghError(rc, load().egh_server_last_error(sv).decode())


class Server:
    """Continuous batching of deblur requests against resident factored Hessian sets
    (egh_server_* in include/egh.h).  Host buffers should be pinned and must stay alive until
    wait() returns for their request."""

    def __init__(self, hbm_budget_bytes, slots=4, max_batch_sources=128, precision=EGH_PREC_FP32):
        cfg = egh_server_config(int(hbm_budget_bytes), int(slots), int(max_batch_sources), int(precision))
        h = _vp()
        _check_server(load().egh_server_create(ctypes.byref(cfg), ctypes.byref(h)), None)
        self.h = h
        self._keep = {}

    def add_set(self, Q, freq_hz, dt, nt_record, max_nt):
        """Q: [nf][nrec][nrec] complex64 host array (Hermitian positive definite)."""
        Q = np.ascontiguousarray(Q, dtype=np.complex64)
        f = np.ascontiguousarray(freq_hz, dtype=np.float64)
        sid = ctypes.c_int32(0)
        _check_server(load().egh_server_add_set(self.h, int(Q.shape[1]), int(f.size), f.ctypes.data_as(_f64p),
                                                float(dt), int(nt_record), int(max_nt), Q.ctypes.data,
                                                ctypes.byref(sid)), self.h)
        return sid.value

    def submit(self, set_id, resid, mult):
        """resid, mult: [ns][nrec][nt_d] float32 host buffers (torch pinned tensors or numpy)."""
        pi, _ = _ptr(resid)
        po, _ = _ptr(mult)
        ns, _, nt_d = resid.shape
        rid = ctypes.c_int64(0)
        _check_server(load().egh_server_submit(self.h, int(set_id), pi, int(ns), int(nt_d), po,
                                               ctypes.byref(rid)), self.h)
        self._keep[rid.value] = (resid, mult)
        return rid.value

    def wait(self, request_id, timeout_s=60.0):
        lat = ctypes.c_double(0.0)
        st = load().egh_server_wait(self.h, int(request_id), float(timeout_s), ctypes.byref(lat))
        if st != EGH_ETIMEOUT:
            # finished or failed: the id is released and no kernel touches the buffers any more
            # (on EGH_ETIMEOUT they stay referenced until the server closes)
            self._keep.pop(request_id, None)
        _check_server(st, self.h)
        return lat.value

    def drain(self, timeout_s=120.0):
        _check_server(load().egh_server_drain(self.h, float(timeout_s)), self.h)

    def stats(self):
        s = egh_server_stats()
        _check_server(load().egh_server_get_stats(self.h, ctypes.byref(s)), self.h)
        return s.as_dict()

    def reset_stats(self):
        _check_server(load().egh_server_reset_stats(self.h), self.h)

    def test_expire_wait(self, count=1):
        _check_server(load().egh_server_test_expire_wait(self.h, int(count)), self.h)

    def hold(self, on=True):
        """Pauses (on) or resumes (off) admission; requests submitted while held queue and are
        packed into batches together when admission resumes."""
        _check_server(load().egh_server_hold(self.h, 1 if on else 0), self.h)

    def close(self):
        if self.h:
            load().egh_server_destroy(self.h)
            self.h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
