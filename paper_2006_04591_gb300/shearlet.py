"""Thin Python binding of libshearlet (include/shearlet.h).

Functions carry the C names and only marshal arguments: torch tensors become
device pointers, the current torch stream becomes the cudaStream_t.  Every
step of the transform runs in the CUDA library; if it is missing or fails to
load, the calls raise -- there is no CPU fallback.

:class:`Bank` is a convenience owner of a bank handle that allocates output
and workspace tensors with torch.
"""

from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from . import _build

SHL_F32, SHL_BF16 = 0, 1
SHL_DUAL_WEIGHTED = 1
SHL_OP_DECOMPOSE, SHL_OP_RECONSTRUCT, SHL_OP_SHRINK = 0, 1, 2
(SHL_OK, SHL_EINVAL, SHL_ENOMEM, SHL_ECUDA, SHL_EUNSUPPORTED, SHL_ETIMEOUT,
 SHL_EDEVICE) = range(7)
HEADER = os.path.join(os.path.dirname(_build.PKG), "include", "shearlet.h")

_lib = None


SHL_ABI_VERSION_PY = 1   # the header's SHL_ABI_VERSION


class ShearletError(RuntimeError):
    def __init__(self, fn, status, detail):
        super().__init__("%s failed: status %d (%s)" % (fn, status, detail))
        self.status = status


def library_path() -> str:
    """The library this process loads: libshearlet.so, or with
    SHL_LIBRARY=checked the bounds-checked build libshearlet_checked.so."""
    return _build.LIB_CHECKED if os.environ.get("SHL_LIBRARY") == "checked" else _build.LIB


def lib():
    """Load the library (built in-tree by ``_build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError("%s is not built: run __graft_entry__.build() "
                           "or python -m paper_2006_04591_gb300._build" % os.path.basename(path))
    L = ctypes.CDLL(path)
    vp, i, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    P = ctypes.POINTER
    sig = {
        "shl_abi_version": (i, []),
        "shl_status_str": (ctypes.c_char_p, [i]),
        "shl_last_error_detail": (ctypes.c_char_p, []),
        "shl_bank_create": (i, [i, i, i, vp, i, i, P(vp)]),
        "shl_bank_create_from_spectra": (i, [i, i, i, vp, vp, i, P(vp)]),
        "shl_bank_create_gpu": (i, [i, i, i, vp, i, i, P(vp)]),
        "shl_bank_create_general": (i, [i, i, i, vp, vp, vp, i, P(vp)]),
        "shl_ray_create": (i, [i, i, i, i, P(vp)]),
        "shl_ray_destroy": (i, [vp]),
        "shl_ray_query": (i, [vp, P(i), P(i), P(i)]),
        "shl_ray_forward": (i, [vp, vp, i, vp, vp]),
        "shl_ray_adjoint": (i, [vp, vp, i, vp, vp]),
        "shl_bank_path": (i, [vp, P(i)]),
        "shl_bank_copy_spectra_imag": (i, [vp, vp]),
        "shl_bank_destroy": (i, [vp]),
        "shl_bank_query": (i, [vp, P(i), P(i), P(i)]),
        "shl_bank_copy_info": (i, [vp, vp, vp, vp, vp]),
        "shl_workspace_size": (i, [vp, i, i, P(sz)]),
        "shl_decompose": (i, [vp, vp, i, vp, i, i, vp, sz, vp]),
        "shl_decompose_masked": (i, [vp, vp, vp, vp, i, vp, i, vp, sz, vp]),
        "shl_decompose_noalloc": (i, [vp, vp, i, vp, i, i, vp]),
        "shl_reconstruct": (i, [vp, vp, i, i, vp, vp, vp, sz, vp]),
        "shl_adjoint": (i, [vp, vp, i, i, vp, vp, vp, sz, vp]),
        "shl_shrink": (i, [vp, vp, vp, vp, i, vp, vp, vp, sz, vp]),
        "shl_subband_absmax": (i, [vp, vp, i, i, i, vp, vp]),
        "shl_iht_thresholds": (i, [vp, vp, i, i, ctypes.c_double, vp, vp]),
        "shl_sync": (i, [vp]),
        "shl_checked_build": (i, []),
        "shl_check_status": (i, [i, P(ctypes.c_uint)]),
        "shl_launch_count": (ctypes.c_longlong, []),
        "shl_profile_enable": (i, [i]),
        "shl_profile_read": (i, [ctypes.c_char_p, sz]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def header_symbols() -> list[str]:
    """Function names declared in include/*.h."""
    inc = os.path.dirname(HEADER)
    names = set()
    for h in sorted(os.listdir(inc)):
        if h.endswith(".h"):
            txt = open(os.path.join(inc, h)).read()
            names |= set(re.findall(r"^[A-Za-z_][\w \*]*?\b(shl_\w+)\s*\(", txt, re.M))
    return sorted(names)


def _check(fn, status):
    if status != 0:
        L = lib()
        raise ShearletError(fn, status, "%s: %s" % (L.shl_status_str(status).decode(),
                                                     L.shl_last_error_detail().decode()))


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream, device):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return ctypes.c_void_p(stream.cuda_stream)


def _dtype_code(dt):
    import torch
    if dt == torch.float32:
        return SHL_F32
    if dt == torch.bfloat16:
        return SHL_BF16
    raise ValueError("coefficients must be float32 or bfloat16, got %s" % dt)


# ------------------------------------------------------------ C-named calls
def shl_bank_create(rows, cols, n_scales, shear_levels=None, full=0, device=0):
    h = ctypes.c_void_p()
    lv = None
    if shear_levels is not None:
        arr = (ctypes.c_int * len(shear_levels))(*shear_levels)
        lv = ctypes.cast(arr, ctypes.c_void_p)
    _check("shl_bank_create", lib().shl_bank_create(rows, cols, n_scales, lv, int(full), device,
                                                    ctypes.byref(h)))
    return h


def shl_bank_create_gpu(rows, cols, n_scales, shear_levels=None, full=0, device=0):
    h = ctypes.c_void_p()
    lv = None
    if shear_levels is not None:
        arr = (ctypes.c_int * len(shear_levels))(*shear_levels)
        lv = ctypes.cast(arr, ctypes.c_void_p)
    _check("shl_bank_create_gpu", lib().shl_bank_create_gpu(rows, cols, n_scales, lv, int(full),
                                                            device, ctypes.byref(h)))
    return h


def shl_bank_create_from_spectra(spectra, idx=None, device=0):
    S = np.ascontiguousarray(spectra, dtype=np.float64)
    K, N, M = S.shape
    ip = None
    if idx is not None:
        I = np.ascontiguousarray(idx, dtype=np.int32)
        ip = I.ctypes.data_as(ctypes.c_void_p)
    h = ctypes.c_void_p()
    _check("shl_bank_create_from_spectra",
           lib().shl_bank_create_from_spectra(N, M, K, S.ctypes.data_as(ctypes.c_void_p), ip,
                                              device, ctypes.byref(h)))
    return h


def shl_bank_create_general(spectra, idx=None, device=0):
    """Bank on the general kernels; ``spectra`` [K, N, M] real or complex
    (Hermitian), natural order."""
    S = np.asarray(spectra)
    K, N, M = S.shape
    re = np.ascontiguousarray(S.real, dtype=np.float64)
    im = np.ascontiguousarray(S.imag, dtype=np.float64) if np.iscomplexobj(S) else None
    ip = None
    if idx is not None:
        I = np.ascontiguousarray(idx, dtype=np.int32)
        ip = I.ctypes.data_as(ctypes.c_void_p)
    h = ctypes.c_void_p()
    _check("shl_bank_create_general",
           lib().shl_bank_create_general(N, M, K, re.ctypes.data_as(ctypes.c_void_p),
                                         None if im is None else im.ctypes.data_as(ctypes.c_void_p),
                                         ip, device, ctypes.byref(h)))
    return h


def shl_bank_path(h):
    g = ctypes.c_int()
    _check("shl_bank_path", lib().shl_bank_path(h, ctypes.byref(g)))
    return g.value


def shl_bank_copy_spectra_imag(h):
    K, N, M = shl_bank_query(h)
    out = np.zeros((K, N, M), np.float64)
    _check("shl_bank_copy_spectra_imag",
           lib().shl_bank_copy_spectra_imag(h, out.ctypes.data_as(ctypes.c_void_p)))
    return out


def shl_bank_destroy(h):
    _check("shl_bank_destroy", lib().shl_bank_destroy(h))


def shl_bank_query(h):
    K, r, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check("shl_bank_query", lib().shl_bank_query(h, ctypes.byref(K), ctypes.byref(r),
                                                  ctypes.byref(c)))
    return K.value, r.value, c.value


def shl_bank_copy_info(h, spectra=True, dual_w=True):
    K, N, M = shl_bank_query(h)
    idx = np.zeros((K, 3), np.int32)
    rms = np.zeros(K, np.float64)
    S = np.zeros((K, N, M), np.float64) if spectra else None
    W = np.zeros((N, M), np.float64) if dual_w else None
    cp = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)
    _check("shl_bank_copy_info", lib().shl_bank_copy_info(h, cp(idx), cp(rms), cp(S), cp(W)))
    return {"idx": idx, "rms": rms, "spectra": S, "dual_w": W}


def shl_workspace_size(h, op, batch):
    n = ctypes.c_size_t()
    _check("shl_workspace_size", lib().shl_workspace_size(h, op, batch, ctypes.byref(n)))
    return n.value


def shl_decompose(h, x, batch, coeffs, dtype, flags, ws, stream=None):
    _check("shl_decompose", lib().shl_decompose(
        h, _ptr(x), batch, _ptr(coeffs), dtype, flags, _ptr(ws), ws.numel() * ws.element_size(),
        _stream(stream, coeffs.device)))


def bank_builder_version() -> int:
    """SHL_BANK_BUILDER_VERSION as the header defines it (part of the bank
    cache key, so that a changed construction never serves stale spectra)."""
    m = re.search(r"#define\s+SHL_BANK_BUILDER_VERSION\s+(\d+)", open(HEADER).read())
    if not m:
        raise RuntimeError("SHL_BANK_BUILDER_VERSION not found in %s" % HEADER)
    return int(m.group(1))


def noalloc_scratch_bytes() -> int:
    """SHL_NOALLOC_SCRATCH_BYTES as the header defines it."""
    txt = open(HEADER).read()
    m = re.search(r"#define\s+SHL_NOALLOC_SCRATCH_BYTES\s+\((\d+)u\s*<<\s*(\d+)\)", txt)
    if not m:
        raise RuntimeError("SHL_NOALLOC_SCRATCH_BYTES not found in %s" % HEADER)
    return int(m.group(1)) << int(m.group(2))


def noalloc_max_batch(rows, cols) -> int:
    """Largest batch shl_decompose_noalloc accepts: the batch's image spectra
    (rounded up to 256 bytes) plus one subband plane must fit the scratch."""
    plane = rows * (cols // 2 + 1) * 8
    cap = noalloc_scratch_bytes()
    b = 0
    while ((((b + 1) * plane + 255) // 256) * 256) + plane <= cap:
        b += 1
    return b


def shl_decompose_noalloc(h, x, batch, coeffs, dtype, flags, stream=None):
    """shl_decompose using the library's fixed scratch instead of a workspace.

    x and coeffs are checked against the bank's shape before the call: x
    float32 with at least batch*rows*cols elements, coeffs of the element
    type `dtype` names with at least batch*K*rows*cols elements, both on a
    CUDA device."""
    import torch
    K, N, M = shl_bank_query(h)
    want_dt = torch.float32 if dtype == SHL_F32 else torch.bfloat16 if dtype == SHL_BF16 else None
    if want_dt is None:
        raise ValueError("dtype must be SHL_F32 or SHL_BF16")
    if not (x.is_cuda and coeffs.is_cuda):
        raise ValueError("x and coeffs must be CUDA tensors")
    if x.dtype != torch.float32 or not x.is_contiguous() or x.numel() < batch * N * M:
        raise ValueError("x must be contiguous float32 with >= batch*rows*cols elements")
    if coeffs.dtype != want_dt or not coeffs.is_contiguous() or coeffs.numel() < batch * K * N * M:
        raise ValueError("coeffs must be contiguous %s with >= batch*K*rows*cols elements" % want_dt)
    _check("shl_decompose_noalloc", lib().shl_decompose_noalloc(
        h, _ptr(x), batch, _ptr(coeffs), dtype, flags, _stream(stream, coeffs.device)))


def shl_iht_thresholds(h, absmax_by_rms, batch, iterations, delta_min, out, stream=None):
    """Inpainting threshold schedule [iterations][batch][K] on the device."""
    _check("shl_iht_thresholds", lib().shl_iht_thresholds(
        h, _ptr(absmax_by_rms), batch, iterations, float(delta_min), _ptr(out),
        _stream(stream, out.device)))


def shl_decompose_masked(h, f_masked, mask, f_est, batch, coeffs, dtype, ws, stream=None):
    _check("shl_decompose_masked", lib().shl_decompose_masked(
        h, _ptr(f_masked), _ptr(mask), _ptr(f_est), batch, _ptr(coeffs), dtype, _ptr(ws),
        ws.numel() * ws.element_size(), _stream(stream, coeffs.device)))


def shl_reconstruct(h, coeffs, dtype, batch, thresh, x_out, ws, stream=None):
    _check("shl_reconstruct", lib().shl_reconstruct(
        h, _ptr(coeffs), dtype, batch, _ptr(thresh), _ptr(x_out), _ptr(ws),
        ws.numel() * ws.element_size(), _stream(stream, coeffs.device)))


def shl_shrink(h, x, mask, f_est, batch, thresh, x_out, ws, stream=None):
    _check("shl_shrink", lib().shl_shrink(
        h, _ptr(x), _ptr(mask), _ptr(f_est), batch, _ptr(thresh), _ptr(x_out), _ptr(ws),
        ws.numel() * ws.element_size(), _stream(stream, ws.device)))


def shl_adjoint(h, coeffs, dtype, batch, thresh, x_out, ws, stream=None):
    _check("shl_adjoint", lib().shl_adjoint(
        h, _ptr(coeffs), dtype, batch, _ptr(thresh), _ptr(x_out), _ptr(ws),
        ws.numel() * ws.element_size(), _stream(stream, coeffs.device)))


def shl_subband_absmax(h, coeffs, dtype, batch, by_rms, out, stream=None):
    _check("shl_subband_absmax", lib().shl_subband_absmax(
        h, _ptr(coeffs), dtype, batch, int(by_rms), _ptr(out), _stream(stream, out.device)))


def shl_checked_build() -> int:
    return int(lib().shl_checked_build())


def shl_check_status(device=0) -> int:
    """Synchronise `device` and read (and clear) the checked build's guard word."""
    w = ctypes.c_uint(0)
    _check("shl_check_status", lib().shl_check_status(int(device), ctypes.byref(w)))
    return int(w.value)


def shl_sync(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    _check("shl_sync", lib().shl_sync(ctypes.c_void_p(s.cuda_stream)))


def shl_launch_count():
    return int(lib().shl_launch_count())


def shl_profile_enable(on):
    _check("shl_profile_enable", lib().shl_profile_enable(int(on)))


def shl_profile_read():
    import json
    buf = ctypes.create_string_buffer(1 << 16)
    _check("shl_profile_read", lib().shl_profile_read(buf, len(buf)))
    return json.loads(buf.value.decode())


# ------------------------------------------------------------- convenience
class Bank:
    """Owner of a filter-bank handle on one CUDA device."""

    def __init__(self, handle, device):
        self.handle = handle
        self.device = device
        self.K, self.rows, self.cols = shl_bank_query(handle)
        info = shl_bank_copy_info(handle, spectra=False, dual_w=False)
        self.idx, self.rms = info["idx"], info["rms"]
        self.general = bool(shl_bank_path(handle))
        self._rms_dev = None

    @classmethod
    def create(cls, rows, cols, n_scales, shear_levels=None, full=False, device=0, on_gpu=False):
        """Build the digital shearlet system; on_gpu=True constructs it on the
        device (shl_bank_create_gpu), else on the host (shl_bank_create)."""
        make = shl_bank_create_gpu if on_gpu else shl_bank_create
        return cls(make(rows, cols, n_scales, shear_levels, full, device), device)

    @classmethod
    def from_spectra(cls, spectra, idx=None, device=0):
        """Real, even spectra [K, N, M] in natural order (N, M in [1, 4096];
        sizes other than powers of two in [16, 2048] use the general kernels)."""
        return cls(shl_bank_create_from_spectra(spectra, idx, device), device)

    @classmethod
    def from_complex_spectra(cls, spectra, idx=None, device=0):
        """Spectra [K, N, M] (complex Hermitian, or real even) on the general
        kernels, whatever the size."""
        return cls(shl_bank_create_general(spectra, idx, device), device)

    def info(self):
        d = shl_bank_copy_info(self.handle)
        if self.general:
            d["spectra_imag"] = shl_bank_copy_spectra_imag(self.handle)
        return d

    # ------------------------------------------------------- disk cache
    @staticmethod
    def cache_key(rows, cols, n_scales, shear_levels=None, full=False):
        """Hex digest identifying a shearlet-system construction."""
        import hashlib
        lv = list(shear_levels) if shear_levels is not None else None
        txt = "shl-bank-v1|%d|%d|%d|%s|%d|abi%d|builder%d" % (
            rows, cols, n_scales, lv, int(bool(full)), SHL_ABI_VERSION_PY, bank_builder_version())
        return hashlib.sha256(txt.encode()).hexdigest()[:24]

    def save(self, path, key=""):
        """Write the bank's float64 spectra (real and imaginary parts), indices
        and cache key to ``path`` (.npz)."""
        d = self.info()
        imag = d.get("spectra_imag", np.zeros(0))
        if not np.any(imag):
            imag = np.zeros(0)          # a real bank stays real
        np.savez(path, key=np.array(key), spectra=d["spectra"], imag=imag, idx=d["idx"],
                 general=np.array(int(self.general)))

    @classmethod
    def load(cls, path, device=0, key=None):
        """Bank from a file written by ``save``; with ``key`` given, the file's
        key must match (else ValueError)."""
        with np.load(path) as z:
            if key is not None and str(z["key"]) != key:
                raise ValueError("bank cache %s holds key %s, not %s" % (path, z["key"], key))
            S, I, idx = z["spectra"], z["imag"], z["idx"]
            general = bool(int(z["general"]))
        if I.size:
            return cls(shl_bank_create_general(S + 1j * I, idx, device), device)
        if general:
            return cls(shl_bank_create_general(S, idx, device), device)
        return cls(shl_bank_create_from_spectra(S, idx, device), device)

    @classmethod
    def cached(cls, cache_dir, rows, cols, n_scales, shear_levels=None, full=False, device=0):
        """``create`` through a directory of saved banks: load the file named by
        the construction's key if present, else build, save and return."""
        import os
        key = cls.cache_key(rows, cols, n_scales, shear_levels, full)
        path = os.path.join(cache_dir, "bank_%s.npz" % key)
        if os.path.exists(path):
            return cls.load(path, device, key)
        b = cls.create(rows, cols, n_scales, shear_levels, full, device)
        os.makedirs(cache_dir, exist_ok=True)
        tmp = "%s.%d.tmp.npz" % (path, os.getpid())     # one writer per file name
        try:
            b.save(tmp, key)
            os.replace(tmp, path)                       # atomic: readers see old or new
        finally:
            if os.path.exists(tmp):                     # save or replace failed
                os.remove(tmp)
        return b

    def close(self):
        if self.handle is not None:
            shl_bank_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def rms_device(self):
        import torch
        if self._rms_dev is None:
            self._rms_dev = torch.tensor(self.rms, dtype=torch.float32,
                                         device="cuda:%d" % self.device)
        return self._rms_dev

    def workspace(self, op, batch):
        import torch
        n = shl_workspace_size(self.handle, op, batch)
        return torch.empty(max(n, 16), dtype=torch.uint8, device="cuda:%d" % self.device)

    def _check_images(self, x):
        """Images are CUDA tensors, or pinned host tensors that the kernels read
        / write over the CPU-GPU link (the C ABI maps them)."""
        if x.dim() != 3 or x.shape[1:] != (self.rows, self.cols):
            raise ValueError("expected [B, %d, %d] images, got %s" % (self.rows, self.cols,
                                                                     tuple(x.shape)))
        if not x.is_contiguous() or not (x.is_cuda or x.is_pinned()):
            raise ValueError("images must be contiguous CUDA or pinned host tensors")

    def _dev(self):
        import torch
        return torch.device("cuda", self.device)

    def decompose(self, x, dtype=None, dual=False, out=None, ws=None):
        import torch
        dtype = dtype or torch.float32
        x = x.contiguous()
        self._check_images(x)
        B = x.shape[0]
        c = out if out is not None else torch.empty((B, self.K, self.rows, self.cols),
                                                    dtype=dtype, device=self._dev())
        ws = ws if ws is not None else self.workspace(SHL_OP_DECOMPOSE, B)
        shl_decompose(self.handle, x, B, c, _dtype_code(c.dtype),
                      SHL_DUAL_WEIGHTED if dual else 0, ws)
        return c

    def decompose_masked(self, f_masked, mask_u8, f_est, dtype=None, out=None, ws=None):
        import torch
        dtype = dtype or torch.float32
        self._check_images(f_masked)
        B = f_masked.shape[0]
        c = out if out is not None else torch.empty((B, self.K, self.rows, self.cols),
                                                    dtype=dtype, device=self._dev())
        ws = ws if ws is not None else self.workspace(SHL_OP_DECOMPOSE, B)
        shl_decompose_masked(self.handle, f_masked, mask_u8, f_est, B, c,
                             _dtype_code(c.dtype), ws)
        return c

    def _rec(self, fn, c, thresh, out, ws):
        import torch
        c = c.contiguous()
        if c.dim() != 4 or c.shape[1:] != (self.K, self.rows, self.cols):
            raise ValueError("expected [B, K, N, M] coefficients, got %s" % (tuple(c.shape),))
        B = c.shape[0]
        x = out if out is not None else torch.empty((B, self.rows, self.cols),
                                                    dtype=torch.float32, device=c.device)
        if thresh is not None:
            thresh = thresh.to(device=c.device, dtype=torch.float32).contiguous()
            if thresh.shape != (B, self.K):
                raise ValueError("thresholds must be [B, K]")
        ws = ws if ws is not None else self.workspace(SHL_OP_RECONSTRUCT, B)
        fn(self.handle, c, _dtype_code(c.dtype), B, thresh, x, ws)
        return x

    def reconstruct(self, c, thresh=None, out=None, ws=None):
        return self._rec(shl_reconstruct, c, thresh, out, ws)

    def adjoint(self, c, thresh=None, out=None, ws=None):
        return self._rec(shl_adjoint, c, thresh, out, ws)

    def shrink(self, x, thresh, mask_u8=None, f_est=None, out=None, ws=None):
        """rec(T_thresh(dec(u))), u = x or mask (x - f_est) + f_est, without
        storing coefficients (shl_shrink)."""
        import torch
        x = x.contiguous()
        self._check_images(x)
        B = x.shape[0]
        thresh = thresh.to(device=self._dev(), dtype=torch.float32).contiguous()
        if thresh.shape != (B, self.K):
            raise ValueError("thresholds must be [B, K]")
        if (mask_u8 is None) != (f_est is None):
            raise ValueError("mask and f_est go together")
        if mask_u8 is not None:
            mask_u8 = mask_u8.contiguous()
            f_est = f_est.contiguous()
            self._check_images(f_est)
        y = out if out is not None else torch.empty(x.shape, dtype=torch.float32,
                                                    device=self._dev())
        ws = ws if ws is not None else self.workspace(SHL_OP_SHRINK, B)
        shl_shrink(self.handle, x, mask_u8, f_est, B, thresh, y, ws)
        return y

    def iht_thresholds(self, absmax_by_rms, iterations, delta_min=0.02, out=None):
        """[iterations, B, K] inpainting thresholds from max |c_i| / RMS_i [B, K]."""
        import torch
        B = absmax_by_rms.shape[0]
        out = out if out is not None else torch.empty((iterations, B, self.K), dtype=torch.float32,
                                                      device=absmax_by_rms.device)
        shl_iht_thresholds(self.handle, absmax_by_rms.contiguous(), B, iterations, delta_min, out)
        return out

    def subband_absmax(self, c, by_rms=False, out=None):
        import torch
        B = c.shape[0]
        out = out if out is not None else torch.empty((B, self.K), dtype=torch.float32,
                                                      device=c.device)
        shl_subband_absmax(self.handle, c.contiguous(), _dtype_code(c.dtype), B, by_rms, out)
        return out
