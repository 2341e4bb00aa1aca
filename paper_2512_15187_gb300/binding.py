"""Thin ctypes binding of libpid.so (argument marshalling only).

The functions named pid_* mirror the C ABI of include/pid.h one to one and take raw
device pointers (ints) and sizes. `Handle` adds the same calls on torch CUDA tensors:
it reads data pointers and strides, allocates the output tensors on the device and
passes the current torch stream. Every computation runs in the library's CUDA kernels;
if libpid.so is missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_int32, c_int64, c_size_t, c_void_p

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libpid.so")

PID_OK, PID_ERR_INVALID_ARG, PID_ERR_DOMAIN, PID_ERR_OOM, PID_ERR_CUDA = 0, 1, 2, 3, 4
PID_ERR_TIMEOUT, PID_ERR_BUSY, PID_ERR_CANCELLED, PID_ERR_UNSUPPORTED = 5, 6, 7, 8
PID_MODE_MEAN, PID_MODE_FULL, PID_MODE_FULL_LINEAR = 0, 1, 2
PID_FP32, PID_BF16, PID_SPLIT_BF16, PID_FP8 = 0, 1, 2, 3
PID_ISO_NORMAL = 0
PID_ISO_UNIFORM = 1
PID_ISO_LEVEL = 2

MODES = {"mean": PID_MODE_MEAN, "full": PID_MODE_FULL, "gram": PID_MODE_FULL,
         "linear": PID_MODE_FULL_LINEAR, "full_linear": PID_MODE_FULL_LINEAR}
PRECISIONS = {"fp32": PID_FP32, "bf16": PID_BF16, "split_bf16": PID_SPLIT_BF16, "fp8": PID_FP8}

EXPORTS = [
    "pid_create", "pid_destroy", "pid_sync", "pid_status_string", "pid_last_error",
    "pid_workspace_bytes", "pid_soft_masks", "pid_mean", "pid_full", "pid_from_fields",
    "pid_batch", "pid_profile_enable", "pid_profile_read", "pid_autotune_enable",
    "pid_mean_noalloc", "pid_serve_start", "pid_serve_stop", "pid_serve_register",
    "pid_serve_update", "pid_serve_unregister", "pid_serve_submit", "pid_serve_wait",
    "pid_serve_stats_get", "pid_serve_stats_reset", "pid_contour_bands", "pid_mean_weighted",
    "pid_spacetime", "pid_depth_from_matrix", "pid_soft_masks_bf16",
    "pid_selftest_wait_timeout", "pid_gram_operands", "pid_serve_cancel",
    "pid_autotune_shapes", "pid_autotune_describe",
]
PID_KERNEL_STREAM, PID_KERNEL_GRAM, PID_KERNEL_FINALIZE, PID_KERNEL_ISO, PID_KERNEL_BANDS = 0, 1, 2, 3, 4
PID_KERNEL_GRAM_SPLIT, PID_KERNEL_GRAM_FP8, PID_KERNEL_OPERANDS, PID_KERNEL_SCALE = 5, 6, 7, 8
BAND_INNER_UNION, BAND_INNER_INTERSECTION, BAND_ALL_UNION, BAND_ALL_INTERSECTION, BAND_MEDIAN = \
    1, 2, 4, 8, 16
KERNEL_KINDS = {"stream": 0, "gram": 1, "finalize": 2, "iso": 3, "bands": 4, "gram_split": 5,
                "gram_fp8": 6, "operands": 7, "scale": 8}


class PidError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"[pid status {status}] {message}")
        self.status = status


class pid_iso(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("superlevel", c_int32), ("mu", c_double), ("sigma", c_double)]


ISO_KINDS = {"normal": PID_ISO_NORMAL, "uniform": PID_ISO_UNIFORM, "level": PID_ISO_LEVEL}


def make_iso(iso) -> "pid_iso":
    """pid_iso from (mu, sigma[, superlevel[, kind]]); kind is "normal" (default), "uniform"
    or "level" (or the PID_ISO_* value)."""
    kind = iso[3] if len(iso) > 3 else "normal"
    kind = ISO_KINDS[kind] if isinstance(kind, str) else int(kind)
    return pid_iso(kind, int(iso[2]) if len(iso) > 2 else 0, float(iso[0]), float(iso[1]))


class pid_options(ctypes.Structure):
    _fields_ = [("mode", c_int32), ("precision", c_int32), ("validate", c_int32),
                ("reserved", c_int32)]


class pid_kernel_stats(ctypes.Structure):
    _fields_ = [("launches", c_int64), ("total_ms", c_double), ("bytes", c_double),
                ("flops", c_double)]


class pid_ensemble(ctypes.Structure):
    _fields_ = [("data", c_void_p), ("N", c_int64), ("M", c_int64), ("ld", c_int64),
                ("w", c_void_p), ("is_field", c_int32), ("reserved", c_int32),
                ("iso", pid_iso), ("opt", pid_options),
                ("depth", c_void_p), ("in_in", c_void_p), ("in_out", c_void_p),
                ("rank", c_void_p), ("mass", c_void_p), ("mean_depth", c_void_p),
                ("P", c_void_p), ("err_est", c_void_p)]


class pid_serve_cfg(ctypes.Structure):
    _fields_ = [("device", c_int32), ("max_inflight", c_int32), ("max_batch", c_int32),
                ("max_queue", c_int32), ("hbm_budget_bytes", c_size_t),
                ("workspace_reserve_bytes", c_size_t), ("max_step_member_cells", c_int64)]


class pid_serve_stats(ctypes.Structure):
    _fields_ = [("submitted", c_int64), ("completed", c_int64), ("failed", c_int64),
                ("steps", c_int64), ("mean_batch", c_double), ("p50_ms", c_double),
                ("p99_ms", c_double), ("max_ms", c_double), ("requests_per_s", c_double),
                ("member_cells_per_s", c_double), ("resident_bytes", c_size_t)]


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libpid.so (raises if it is missing: there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libpid.so not found at {path}; build it with "
                           "`python -m paper_2512_15187_gb300.build`")
    lib = ctypes.CDLL(path)
    P = c_void_p
    sig = {
        "pid_create": ([POINTER(c_void_p), c_int, c_size_t], c_int),
        "pid_destroy": ([P], c_int),
        "pid_sync": ([P, P], c_int),
        "pid_status_string": ([c_int], c_char_p),
        "pid_last_error": ([P], c_char_p),
        "pid_workspace_bytes": ([P], c_size_t),
        "pid_soft_masks": ([P, P, c_int64, c_int64, c_int64, POINTER(pid_iso), P, c_int64, P], c_int),
        "pid_soft_masks_bf16": ([P, P, c_int64, c_int64, c_int64, POINTER(pid_iso), P, c_int64, P],
                                c_int),
        "pid_selftest_wait_timeout": ([P, ctypes.c_double, P], c_int),
        "pid_contour_bands": ([P, P, c_int64, c_int64, c_int64, POINTER(pid_iso), P, ctypes.c_double,
                               ctypes.c_double, P, P], c_int),
        "pid_mean": ([P, P, c_int64, c_int64, c_int64, P, P, P, P, P, P], c_int),
        "pid_full": ([P, P, c_int64, c_int64, c_int64, P, POINTER(pid_options), P, P, P, P, P, P, P],
                     c_int),
        "pid_from_fields": ([P, P, c_int64, c_int64, c_int64, P, POINTER(pid_iso),
                             POINTER(pid_options), P, P, P, P, P], c_int),
        "pid_mean_weighted": ([P, P, c_int64, c_int64, c_int64, P, POINTER(pid_iso), P, P, P, P, P,
                               P], c_int),
        "pid_batch": ([P, POINTER(pid_ensemble), c_int32, P], c_int),
        "pid_depth_from_matrix": ([P, P, c_int64, c_int64, P, P, P, P, P, P], c_int),
        "pid_spacetime": ([P, P, c_int32, c_int64, c_int64, c_int64, P, POINTER(pid_iso),
                           POINTER(pid_options), P, P, P, P, P, P, P], c_int),
        "pid_profile_enable": ([P, c_int], c_int),
        "pid_profile_read": ([P, c_int, POINTER(pid_kernel_stats)], c_int),
        "pid_autotune_enable": ([P, c_int, POINTER(c_int32)], c_int),
        "pid_autotune_shapes": ([P, POINTER(pid_ensemble), c_int32, P], c_int),
        "pid_autotune_describe": ([P, ctypes.c_char_p, c_int32], c_int32),
        "pid_mean_noalloc": ([P, c_int64, c_int64, c_int64, P, P, P, P, P, P, P], c_int),
        "pid_serve_start": ([POINTER(c_void_p), POINTER(pid_serve_cfg)], c_int),
        "pid_serve_stop": ([P], c_int),
        "pid_serve_cancel": ([P], c_int),
        "pid_gram_operands": ([c_int32, c_int64, c_int32, POINTER(c_int32)], c_int),
        "pid_serve_register": ([P, P, c_int64, c_int64, c_int64, P, c_int32, POINTER(pid_iso),
                                c_int32, POINTER(c_int64)], c_int),
        "pid_serve_update": ([P, c_int64, P], c_int),
        "pid_serve_unregister": ([P, c_int64], c_int),
        "pid_serve_submit": ([P, c_int64, POINTER(pid_options), POINTER(ctypes.c_uint64)], c_int),
        "pid_serve_wait": ([P, ctypes.c_uint64, c_int64, P, P, P, P, P], c_int),
        "pid_serve_stats_get": ([P, POINTER(pid_serve_stats)], c_int),
        "pid_serve_stats_reset": ([P], c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(h, status: int):
    if status != PID_OK:
        lib = load()
        msg = lib.pid_last_error(h).decode() if h else lib.pid_status_string(status).decode()
        raise PidError(status, msg or lib.pid_status_string(status).decode())


# --- raw C-ABI mirrors (device pointers as ints) -------------------------------------------

def pid_create(device: int = 0, hbm_budget_bytes: int = 0):
    h = c_void_p()
    st = load().pid_create(ctypes.byref(h), device, hbm_budget_bytes)
    if st != PID_OK:
        raise PidError(st, load().pid_status_string(st).decode())
    return h


def pid_destroy(h):
    _check(None, load().pid_destroy(h))


def pid_sync(h, stream=None):
    _check(h, load().pid_sync(h, stream))


def pid_contour_bands(h, data, N, M, ld, iso, rank, tau, inner_fraction, bands, stream=None):
    _check(h, load().pid_contour_bands(h, data, N, M, ld, None if iso is None else ctypes.byref(iso),
                                       rank, float(tau), float(inner_fraction), bands, stream))


def pid_soft_masks(h, F, N, M, ld, iso: pid_iso, U_out, ld_out, stream=None):
    _check(h, load().pid_soft_masks(h, F, N, M, ld, ctypes.byref(iso), U_out, ld_out, stream))


def pid_mean(h, U, N, M, ld, w, depth, in_in, in_out, rank, stream=None):
    _check(h, load().pid_mean(h, U, N, M, ld, w, depth, in_in, in_out, rank, stream))


def pid_full(h, U, N, M, ld, w, opt: pid_options, depth, in_in, in_out, rank, P, err_est,
             stream=None):
    _check(h, load().pid_full(h, U, N, M, ld, w, ctypes.byref(opt) if opt else None, depth, in_in,
                              in_out, rank, P, err_est, stream))


def pid_from_fields(h, F, N, M, ld, w, iso: pid_iso, opt: pid_options, depth, in_in, in_out, rank,
                    stream=None):
    _check(h, load().pid_from_fields(h, F, N, M, ld, w, ctypes.byref(iso),
                                     ctypes.byref(opt) if opt else None, depth, in_in, in_out,
                                     rank, stream))


def pid_mean_weighted(h, data, N, M, ld, w, iso, member_weights, depth, in_in, in_out, rank,
                      stream=None):
    _check(h, load().pid_mean_weighted(h, data, N, M, ld, w,
                                       None if iso is None else ctypes.byref(iso), member_weights,
                                       depth, in_in, in_out, rank, stream))


def pid_spacetime(h, steps, N, M, ld, w, iso, opt, depth, in_in, in_out, rank, P, err_est,
                  stream=None):
    arr = (c_void_p * len(steps))(*steps)
    _check(h, load().pid_spacetime(h, arr, len(steps), N, M, ld, w,
                                   None if iso is None else ctypes.byref(iso),
                                   ctypes.byref(opt) if opt else None, depth, in_in, in_out,
                                   rank, P, err_est, stream))


def pid_depth_from_matrix(h, P_, N, ldp, labels, depth, in_in, in_out, rank, stream=None):
    _check(h, load().pid_depth_from_matrix(h, P_, N, ldp, labels, depth, in_in, in_out, rank,
                                           stream))


def pid_profile_enable(h, enable: bool):
    _check(h, load().pid_profile_enable(h, int(enable)))


def pid_profile_read(h, kind: int) -> pid_kernel_stats:
    st = pid_kernel_stats()
    _check(h, load().pid_profile_read(h, kind, ctypes.byref(st)))
    return st


def pid_autotune_enable(h, enable: bool) -> int:
    n = c_int32(0)
    _check(h, load().pid_autotune_enable(h, int(enable), ctypes.byref(n)))
    return int(n.value)


_NOALLOC_STATUS = {
    PID_ERR_INVALID_ARG: "N, M or ld out of range (N >= 1, M >= 1, ld >= M), a null U, or no output",
    PID_ERR_UNSUPPORTED: "N above 512, or more per-chunk partials than the fixed 4 MiB scratch holds",
    PID_ERR_CUDA: "the one-time device set-up or a kernel launch failed",
}


def pid_mean_noalloc(U, N, M, ld, w, depth, in_in, in_out, rank, device_status=None,
                     stream=None):
    """PID-mean through the allocation-free entry point (no handle; fixed internal scratch).
    It reports status codes only (there is no handle for pid_last_error): the error text
    says what each code means for this call."""
    st = load().pid_mean_noalloc(U, N, M, ld, w, depth, in_in, in_out, rank, device_status,
                                 stream)
    if st != PID_OK:
        raise PidError(st, "pid_mean_noalloc: " + _NOALLOC_STATUS.get(
            st, load().pid_status_string(st).decode()))


def pid_gram_operands(precision, cells: int, want_matrix: bool) -> int:
    """The operand precision (PID_BF16, PID_SPLIT_BF16 or PID_FP8) a Gram request runs with."""
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    out = c_int32(-1)
    _check(None, load().pid_gram_operands(prec, int(cells), int(bool(want_matrix)),
                                          ctypes.byref(out)))
    return int(out.value)


def pid_batch(h, ensembles, stream=None):
    arr = (pid_ensemble * len(ensembles))(*ensembles)
    _check(h, load().pid_batch(h, arr, len(ensembles), stream))


# --- torch tensor convenience -----------------------------------------------------------------

def _ptr(t):
    return None if t is None else t.data_ptr()


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return c_void_p(s.cuda_stream)


def _check_matrix(x, name):
    import torch
    if x.dim() != 2 or x.dtype != torch.float32 or not x.is_cuda or x.stride(1) != 1:
        raise ValueError(f"{name} must be a 2-D float32 CUDA tensor with unit cell stride")
    return x.shape[0], x.shape[1], x.stride(0)


def _weights(w, M, device):
    """Device pointer of the cell measures w (float32 CUDA [M], contiguous), or None."""
    import torch
    if w is None:
        return None
    if (w.dtype != torch.float32 or not w.is_cuda or w.device != device or
            w.numel() != M or (w.dim() == 1 and w.stride(0) != 1) or not w.is_contiguous()):
        raise ValueError("w must be a contiguous float32 CUDA tensor of M cell measures on "
                         "the data's device")
    return w.data_ptr()


class Handle:
    """A libpid handle bound to one CUDA device; methods take and return torch tensors."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.device = device
        self.h = pid_create(device, hbm_budget_bytes)

    def close(self):
        if self.h:
            pid_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync(self, stream=None):
        pid_sync(self.h, _stream(stream))

    def autotune(self, enable: bool = True) -> int:
        return pid_autotune_enable(self.h, enable)

    def profile(self, enable: bool = True):
        pid_profile_enable(self.h, enable)

    def profile_read(self):
        """{kind: {launches, total_ms, bytes, flops}} for every kernel kind."""
        out = {}
        for name, k in KERNEL_KINDS.items():
            st = pid_profile_read(self.h, k)
            out[name] = {"launches": int(st.launches), "total_ms": float(st.total_ms),
                         "bytes": float(st.bytes), "flops": float(st.flops)}
        return out

    def workspace_bytes(self) -> int:
        return int(load().pid_workspace_bytes(self.h))

    def _outputs(self, N, want_P=False, extras=False, want_err=False):
        import torch
        dev = torch.device("cuda", self.device)
        o = {k: torch.empty(N, dtype=torch.float64, device=dev) for k in ("depth", "in_in", "in_out")}
        o["rank"] = torch.empty(N, dtype=torch.int32, device=dev)
        if want_P:
            o["P"] = torch.empty((N, N), dtype=torch.float64, device=dev)
        if want_P or want_err:
            o["err_est"] = torch.empty(1, dtype=torch.float64, device=dev)
        if extras:
            o["mass"] = torch.empty(N, dtype=torch.float64, device=dev)
            o["mean_depth"] = torch.empty(N, dtype=torch.float64, device=dev)
        return o

    def contour_bands(self, data, rank, tau, inner_fraction=0.5, iso=None, out=None, stream=None):
        """Band flags per cell (uint8 [M], bits BAND_*) of the contour boxplot of the members
        of `data` ([N][ld] soft masks, or fields with iso=(mu, sigma, superlevel)), ordered by
        `rank` (int32 [N] on the device, 0 = deepest), binarised at u > tau."""
        import torch
        N, M, ld = _check_matrix(data, "data")
        if rank.dtype != torch.int32 or not rank.is_cuda or rank.numel() != N:
            raise ValueError("rank must be an int32 CUDA tensor with one entry per member")
        if out is None:
            out = torch.empty(M, dtype=torch.uint8, device=data.device)
        iso_s = None if iso is None else make_iso(iso)
        pid_contour_bands(self.h, data.data_ptr(), N, M, ld, iso_s, rank.data_ptr(), tau,
                          inner_fraction, out.data_ptr(), _stream(stream))
        return out

    def soft_masks(self, F, mu, sigma, superlevel=False, out=None, stream=None, kind="normal",
                   dtype=None):
        """Soft masks of the fields F; dtype torch.float32 (default) or torch.bfloat16."""
        import torch
        N, M, ld = _check_matrix(F, "F")
        dtype = dtype if dtype is not None else (out.dtype if out is not None else torch.float32)
        if dtype not in (torch.float32, torch.bfloat16):
            raise ValueError("soft masks are float32 or bfloat16")
        if out is None:
            out = torch.empty((N, M), dtype=dtype, device=F.device)
        if out.dtype != dtype or not out.is_cuda or out.dim() != 2 or out.stride(1) != 1 or \
                out.shape[0] != N or out.shape[1] < M:
            raise ValueError("out must be an [N, >= M] CUDA tensor of the requested dtype")
        iso = make_iso((mu, sigma, superlevel, kind))
        fn = load().pid_soft_masks_bf16 if dtype == torch.bfloat16 else load().pid_soft_masks
        _check(self.h, fn(self.h, F.data_ptr(), N, M, ld, ctypes.byref(iso), out.data_ptr(),
                          out.stride(0), _stream(stream)))
        return out

    def mean(self, U, w=None, stream=None):
        N, M, ld = _check_matrix(U, "U")
        o = self._outputs(N)
        pid_mean(self.h, U.data_ptr(), N, M, ld, _weights(w, M, U.device), o["depth"].data_ptr(),
                 o["in_in"].data_ptr(), o["in_out"].data_ptr(), o["rank"].data_ptr(),
                 _stream(stream))
        return o

    def mean_weighted(self, data, member_weights, w=None, iso=None, stream=None):
        """PID-mean against the weighted mean contour sum_j r_j u_j / sum_j r_j; data are soft
        masks, or fields with iso=(mu, sigma[, superlevel[, kind]]); member_weights is a
        float64 CUDA tensor [N]."""
        import torch
        N, M, ld = _check_matrix(data, "data")
        r = member_weights
        if r.dtype != torch.float64 or not r.is_cuda or r.numel() != N or not r.is_contiguous():
            raise ValueError("member_weights must be a contiguous float64 CUDA tensor [N]")
        o = self._outputs(N)
        pid_mean_weighted(self.h, data.data_ptr(), N, M, ld, _weights(w, M, data.device),
                          None if iso is None else make_iso(iso), r.data_ptr(),
                          o["depth"].data_ptr(), o["in_in"].data_ptr(), o["in_out"].data_ptr(),
                          o["rank"].data_ptr(), _stream(stream))
        return o

    def spacetime(self, steps, w=None, iso=None, mode="mean", precision="fp32", want_P=False,
                  validate=False, stream=None):
        """4D PID over the time steps `steps` (a list of [N][ld] CUDA tensors of one shape):
        the cells (x, t) of all steps form one ensemble; the steps are not copied."""
        if not steps:
            raise ValueError("need at least one time step")
        N, M, ld = _check_matrix(steps[0], "steps[0]")
        for t, S in enumerate(steps):
            if _check_matrix(S, f"steps[{t}]") != (N, M, ld):
                raise ValueError("every time step needs the shape and row stride of steps[0]")
        gram = MODES[mode] == PID_MODE_FULL and PRECISIONS[precision] != PID_FP32
        o = self._outputs(N, want_P=want_P and gram)
        opt = pid_options(MODES[mode], PRECISIONS[precision], int(validate), 0)
        pid_spacetime(self.h, [S.data_ptr() for S in steps], N, M, ld,
                      _weights(w, M, steps[0].device),
                      None if iso is None else make_iso(iso), opt, o["depth"].data_ptr(),
                      o["in_in"].data_ptr(), o["in_out"].data_ptr(), o["rank"].data_ptr(),
                      _ptr(o.get("P")), _ptr(o.get("err_est")), _stream(stream))
        return o

    def depth_from_matrix(self, P, labels=None, stream=None):
        """Depths from an inclusion matrix P (float64 CUDA [N][ldp], P[i, j] = u_i subset_p
        u_j), within the groups of `labels` (int32 CUDA [N]) or over all members."""
        import torch
        if P.dtype != torch.float64 or not P.is_cuda or P.dim() != 2 or P.stride(1) != 1:
            raise ValueError("P must be a float64 CUDA matrix with unit column stride")
        N = P.shape[0]
        if P.shape[1] != N:
            raise ValueError("P must be square")
        if labels is not None and (labels.dtype != torch.int32 or not labels.is_cuda or
                                   labels.numel() != N or not labels.is_contiguous()):
            raise ValueError("labels must be a contiguous int32 CUDA tensor with one entry per member")
        o = self._outputs(N)
        pid_depth_from_matrix(self.h, P.data_ptr(), N, P.stride(0), _ptr(labels),
                              o["depth"].data_ptr(), o["in_in"].data_ptr(),
                              o["in_out"].data_ptr(), o["rank"].data_ptr(), _stream(stream))
        return o

    def full(self, U, w=None, mode="linear", precision="fp32", want_P=False, validate=False,
             stream=None, want_err=False):
        """Full PID; want_P returns the inclusion matrix P, want_err (or want_P) the Gram's
        raw error estimate err_est (Gram modes only)."""
        N, M, ld = _check_matrix(U, "U")
        gram = MODES[mode] == PID_MODE_FULL and PRECISIONS[precision] != PID_FP32
        o = self._outputs(N, want_P=want_P and gram, want_err=want_err and gram)
        opt = pid_options(MODES[mode], PRECISIONS[precision], int(validate), 0)
        pid_full(self.h, U.data_ptr(), N, M, ld, _weights(w, M, U.device), opt,
                 o["depth"].data_ptr(),
                 o["in_in"].data_ptr(), o["in_out"].data_ptr(), o["rank"].data_ptr(),
                 _ptr(o.get("P")), _ptr(o.get("err_est")), _stream(stream))
        return o

    def from_fields(self, F, mu, sigma, superlevel=False, w=None, mode="mean", precision="fp32",
                    validate=False, stream=None, kind="normal"):
        N, M, ld = _check_matrix(F, "F")
        o = self._outputs(N)
        iso = make_iso((mu, sigma, superlevel, kind))
        opt = pid_options(MODES[mode], PRECISIONS[precision], int(validate), 0)
        pid_from_fields(self.h, F.data_ptr(), N, M, ld, _weights(w, M, F.device), iso, opt,
                        o["depth"].data_ptr(),
                        o["in_in"].data_ptr(), o["in_out"].data_ptr(), o["rank"].data_ptr(),
                        _stream(stream))
        return o

    def autotune_shapes(self, items, stream=None):
        """Time the shape-dependent tile choices (streaming tile class, Gram cell chunk) on
        the ensembles of `items` (as for batch) and keep the fastest per shape."""
        ens, _ = self._records(items, None)
        arr = (pid_ensemble * len(ens))(*ens)
        _check(self.h, load().pid_autotune_shapes(self.h, arr, len(ens), _stream(stream)))

    def autotune_describe(self) -> str:
        n = load().pid_autotune_describe(self.h, None, 0)
        buf = ctypes.create_string_buffer(max(1, n + 1))
        load().pid_autotune_describe(self.h, buf, n + 1)
        return buf.value.decode()

    def _records(self, items, outs):
        reuse = outs is not None
        if reuse and len(outs) != len(items):
            raise ValueError("outs must come from a call with the same items")
        ens, new_outs = [], []
        for idx, it in enumerate(items):
            x = it["data"]
            N, M, ld = _check_matrix(x, "data")
            mode = MODES[it.get("mode", "mean")]
            prec = PRECISIONS[it.get("precision", "fp32")]
            gram = mode == PID_MODE_FULL and prec != PID_FP32
            o = outs[idx] if reuse else self._outputs(N, want_P=it.get("want_P", False) and gram,
                                                      extras=True)
            iso = it.get("iso")
            e = pid_ensemble()
            e.data, e.N, e.M, e.ld = x.data_ptr(), N, M, ld
            e.w = _weights(it.get("w"), M, x.device)
            e.is_field = int(iso is not None)
            if iso is not None:
                e.iso = make_iso(iso)
            e.opt = pid_options(mode, prec, int(it.get("validate", False)), 0)
            for k in ("depth", "in_in", "in_out", "rank", "mass", "mean_depth", "P", "err_est"):
                setattr(e, k, _ptr(o.get(k)))
            ens.append(e)
            new_outs.append(o)
        return ens, new_outs

    def batch(self, items, stream=None, outs=None):
        """items: list of dicts with keys data (tensor), w, iso=(mu, sigma, superlevel) or None,
        mode, precision, want_P. Returns a list of output dicts (with mass and mean_depth).
        `outs`: the list a previous call returned for the same items, written again in place
        (the same records then replay the batch's recorded graph)."""
        ens, new_outs = self._records(items, outs)
        pid_batch(self.h, ens, _stream(stream))
        return new_outs


# --- serving --------------------------------------------------------------------------------

class Server:
    """Continuous-batching depth server (pid_serve_*): resident ensembles, queued requests."""

    def __init__(self, device=0, max_inflight=2, max_batch=32, max_queue=4096,
                 hbm_budget_bytes=0, workspace_reserve_bytes=0, max_step_member_cells=0):
        cfg = pid_serve_cfg(device, max_inflight, max_batch, max_queue, hbm_budget_bytes,
                            workspace_reserve_bytes, max_step_member_cells)
        self.s = c_void_p()
        st = load().pid_serve_start(ctypes.byref(self.s), ctypes.byref(cfg))
        if st != PID_OK:
            raise PidError(st, load().pid_status_string(st).decode())

    def _chk(self, st):
        if st != PID_OK:
            raise PidError(st, load().pid_status_string(st).decode())

    def cancel(self):
        """Stop taking requests: queued ones end cancelled, running steps finish, and waits
        return. The server stays valid (waits and stats still work) until stop()."""
        if self.s:
            self._chk(load().pid_serve_cancel(self.s))

    def stop(self):
        if self.s:
            self._chk(load().pid_serve_stop(self.s))
            self.s = None

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass

    def register(self, data, w=None, iso=None, copy=None):
        """data: numpy float32 [N, M] (copied to the device) or a torch CUDA tensor (adopted)."""
        import numpy as np
        ens = ctypes.c_int64(0)
        is_dev = hasattr(data, "is_cuda") and data.is_cuda
        if copy is None:
            copy = not is_dev
        if is_dev:
            if copy:
                raise ValueError("copy=True takes host (numpy) data; device tensors are adopted")
            N, M, ld = _check_matrix(data, "data")
            dptr = data.data_ptr()
            wptr = _weights(w, M, data.device)
            keep = (data, w)
        else:
            data = np.ascontiguousarray(data, dtype=np.float32)
            N, M = data.shape
            ld = M
            dptr = data.ctypes.data
            w = None if w is None else np.ascontiguousarray(w, dtype=np.float32)
            wptr = None if w is None else w.ctypes.data
            keep = None
        iso_s = make_iso(iso) if iso else pid_iso()
        self._chk(load().pid_serve_register(self.s, dptr, N, M, ld, wptr, int(iso is not None),
                                            ctypes.byref(iso_s), int(bool(copy)),
                                            ctypes.byref(ens)))
        if keep is not None:
            self.__dict__.setdefault("_keep", {})[ens.value] = keep
        return ens.value

    def update(self, ens_id, data_host):
        import numpy as np
        data_host = np.ascontiguousarray(data_host, dtype=np.float32)
        self._chk(load().pid_serve_update(self.s, ens_id, data_host.ctypes.data))

    def unregister(self, ens_id):
        self._chk(load().pid_serve_unregister(self.s, ens_id))
        self.__dict__.get("_keep", {}).pop(ens_id, None)

    def submit(self, ens_id, mode="mean", precision="fp32"):
        t = ctypes.c_uint64(0)
        opt = pid_options(MODES[mode], PRECISIONS[precision], 0, 0)
        self._chk(load().pid_serve_submit(self.s, ens_id, ctypes.byref(opt), ctypes.byref(t)))
        return t.value

    def wait(self, ticket, N, timeout_ms=-1):
        """Returns a dict of numpy arrays (depth, in_in, in_out, rank, mean_depth)."""
        import numpy as np
        out = {k: np.empty(N, dtype=np.float64) for k in ("depth", "in_in", "in_out", "mean_depth")}
        out["rank"] = np.empty(N, dtype=np.int32)
        st = load().pid_serve_wait(self.s, ticket, timeout_ms, out["depth"].ctypes.data,
                                   out["in_in"].ctypes.data, out["in_out"].ctypes.data,
                                   out["rank"].ctypes.data, out["mean_depth"].ctypes.data)
        self._chk(st)
        return out

    def stats(self):
        st = pid_serve_stats()
        self._chk(load().pid_serve_stats_get(self.s, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in pid_serve_stats._fields_}

    def reset_stats(self):
        self._chk(load().pid_serve_stats_reset(self.s))
