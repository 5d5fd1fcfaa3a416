"""ctypes binding of the C ABI declared in include/ngdbf.h.

The functions keep the C names and only marshal arguments; every step of the
decode runs in the CUDA library ``libngdbf.so``.  There is no CPU fallback:
loading fails loudly when the library has not been built, and the decode
functions need CUDA device pointers (torch tensors on the GPU work).
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from ._build import LIB_PATH, ROOT

NGDBF_OK = 0
NGDBF_ERR_INVALID_ARG = 1
NGDBF_ERR_OOM = 2
NGDBF_ERR_CUDA = 3
NGDBF_ERR_UNSUPPORTED = 4
NGDBF_ERR_TIMEOUT = 5
NGDBF_ADAPT = 1
NGDBF_SMOOTH = 2
NGDBF_SINGLE = 4
NGDBF_UNIFORM = 8
NGDBF_FP32 = 0
NGDBF_FP16 = 1
NGDBF_FIX = 2
NGDBF_FIXACC = 3
NGDBF_MAX_T = 511
NGDBF_MAX_WINDOW = 126
NGDBF_NOALLOC_SCRATCH_BYTES = 40 << 20

HEADER = os.path.join(ROOT, "include", "ngdbf.h")


class NgdbfError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"ngdbf status {status}: {message}")
        self.status = status


class ngdbf_params(ctypes.Structure):
    _fields_ = [("w", ctypes.c_float), ("theta", ctypes.c_float), ("eta", ctypes.c_float),
                ("lambda_", ctypes.c_float), ("y_max", ctypes.c_float),
                ("t_max", ctypes.c_int32), ("smooth_window", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("q_bits", ctypes.c_int32)]


class ngdbf_job(ctypes.Structure):
    _fields_ = [("code", ctypes.c_void_p), ("y", ctypes.c_void_p), ("n_frames", ctypes.c_int64),
                ("sigma", ctypes.c_float), ("params", ngdbf_params), ("frame_offset", ctypes.c_uint64),
                ("bits", ctypes.c_void_p), ("iters", ctypes.c_void_p), ("pass_", ctypes.c_void_p)]


NGDBF_BATCH_TUNE = 1
NGDBF_BATCH_GRAPH = 2


class ngdbf_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("frames", ctypes.c_int64), ("peak_bytes_in_use", ctypes.c_int64),
                ("peak_requests_on_device", ctypes.c_int32), ("admitted_into_running", ctypes.c_int32)]


class ngdbf_host_stats(ctypes.Structure):
    _fields_ = [("chunks", ctypes.c_int32), ("reserved", ctypes.c_int32), ("h2d_bytes", ctypes.c_int64),
                ("d2h_bytes", ctypes.c_int64), ("h2d_ms", ctypes.c_double), ("kernel_ms", ctypes.c_double),
                ("d2h_ms", ctypes.c_double), ("wall_ms", ctypes.c_double)]


class ngdbf_launch_info(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_int32), ("block", ctypes.c_int32), ("smem_bytes", ctypes.c_int32),
                ("state_in_smem", ctypes.c_int32), ("kernels", ctypes.c_int32),
                ("sm_count", ctypes.c_int32), ("tables_in_smem", ctypes.c_int32), ("cluster", ctypes.c_int32),
                ("split_min_n", ctypes.c_int32)]


def make_params(w=0.75, theta=-0.9, eta=0.96, lam=1.0, y_max=2.5, t_max=100, smooth_window=64,
                variant=0, precision=NGDBF_FP32, q_bits=0) -> ngdbf_params:
    return ngdbf_params(w, theta, eta, lam, y_max, t_max, smooth_window, variant, precision, q_bits)


_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Loads libngdbf.so; raises if it is missing (no fallback exists)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA decoder library not built: {p} is missing "
                           "(run __graft_entry__.build() or paper_1402_2773_gb300._build.build_cuda())")
    lib = ctypes.CDLL(p)
    vp = ctypes.c_void_p
    i32p = ctypes.POINTER(ctypes.c_int32)
    lib.ngdbf_code_create.argtypes = [ctypes.c_int32, ctypes.c_int32, i32p, i32p, ctypes.POINTER(vp)]
    lib.ngdbf_code_destroy.argtypes = [vp]
    lib.ngdbf_code_info.argtypes = [vp, i32p, i32p, i32p, i32p]
    lib.ngdbf_decode.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_float, ctypes.POINTER(ngdbf_params),
                                 ctypes.c_uint64, ctypes.c_uint64, vp, vp, vp, vp]
    lib.ngdbf_decode_host.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_float,
                                      ctypes.POINTER(ngdbf_params), ctypes.c_uint64, ctypes.c_uint64,
                                      vp, vp, vp, ctypes.c_int64]
    lib.ngdbf_decode_noalloc.argtypes = lib.ngdbf_decode.argtypes
    lib.ngdbf_decode_plain.argtypes = lib.ngdbf_decode.argtypes
    lib.ngdbf_decode_trace.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_float, ctypes.POINTER(ngdbf_params),
                                       ctypes.c_uint64, ctypes.c_uint64, vp, vp, vp, ctypes.c_int64, vp, vp, vp]
    lib.ngdbf_batch_create.argtypes = [ctypes.POINTER(ngdbf_job), ctypes.c_int32, ctypes.c_uint64,
                                       ctypes.c_int32, vp, ctypes.POINTER(vp)]
    lib.ngdbf_batch_launch.argtypes = [vp, vp]
    lib.ngdbf_batch_shape.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ngdbf_launch_info)]
    lib.ngdbf_batch_use_shape.argtypes = [vp, ctypes.c_int32]
    lib.ngdbf_batch_destroy.argtypes = [vp]
    lib.ngdbf_server_create.argtypes = [ctypes.c_size_t, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                        ctypes.POINTER(vp)]
    lib.ngdbf_server_submit.argtypes = [vp, vp, vp, ctypes.c_int64, ctypes.c_float, ctypes.POINTER(ngdbf_params),
                                        ctypes.c_uint64, vp, vp, vp, ctypes.POINTER(ctypes.c_uint64)]
    lib.ngdbf_server_poll.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_int32), ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
    lib.ngdbf_server_wait.argtypes = [vp, ctypes.c_double]
    lib.ngdbf_server_get_stats.argtypes = [vp, ctypes.POINTER(ngdbf_server_stats)]
    lib.ngdbf_server_destroy.argtypes = [vp]
    lib.ngdbf_gaussian_range.argtypes = [ctypes.c_uint32, ctypes.c_uint32, vp, vp]
    lib.ngdbf_generator_table.argtypes = [ctypes.POINTER(ctypes.c_float)]
    lib.ngdbf_mix_probe.argtypes = [ctypes.c_int32, vp, ctypes.POINTER(ctypes.c_int64), vp]
    lib.ngdbf_pool_usage.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    lib.ngdbf_host_alloc.argtypes = [ctypes.c_size_t, ctypes.POINTER(vp)]
    lib.ngdbf_host_free.argtypes = [vp]
    lib.ngdbf_host_huge_page_bytes.argtypes = [ctypes.POINTER(ctypes.c_int64)]
    lib.ngdbf_host_block_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    lib.ngdbf_set_host_copy_mode.argtypes = [ctypes.c_int32]
    lib.ngdbf_get_host_copy_mode.argtypes = [ctypes.POINTER(ctypes.c_int32)]
    lib.ngdbf_last_launch.argtypes = [ctypes.POINTER(ngdbf_launch_info)]
    lib.ngdbf_last_host_stats.argtypes = [ctypes.POINTER(ngdbf_host_stats)]
    lib.ngdbf_last_error.argtypes = []
    lib.ngdbf_last_error.restype = ctypes.c_char_p
    for fn in ("ngdbf_code_create", "ngdbf_code_destroy", "ngdbf_code_info", "ngdbf_decode",
               "ngdbf_decode_host", "ngdbf_decode_noalloc", "ngdbf_decode_trace", "ngdbf_last_launch", "ngdbf_batch_create",
               "ngdbf_batch_launch", "ngdbf_batch_destroy", "ngdbf_server_create", "ngdbf_server_submit",
               "ngdbf_server_poll", "ngdbf_server_wait", "ngdbf_server_get_stats", "ngdbf_server_destroy",
               "ngdbf_gaussian_range", "ngdbf_pool_usage", "ngdbf_last_host_stats", "ngdbf_mix_probe",
               "ngdbf_generator_table", "ngdbf_batch_shape", "ngdbf_batch_use_shape", "ngdbf_decode_plain",
               "ngdbf_host_alloc", "ngdbf_host_free", "ngdbf_host_huge_page_bytes", "ngdbf_host_block_info",
               "ngdbf_set_host_copy_mode", "ngdbf_get_host_copy_mode"):
        getattr(lib, fn).restype = ctypes.c_int
    if path is None:
        _lib = lib
    return lib


def declared_functions() -> list[str]:
    """Names of the functions include/ngdbf.h declares."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ngdbf_[a-z_0-9]+)\s*\(", src)))


def _check(lib, status: int) -> None:
    if status != NGDBF_OK:
        raise NgdbfError(status, lib.ngdbf_last_error().decode())


# --- C-named entry points (argument marshalling only) --------------------------------------------

def ngdbf_last_error() -> str:
    return load().ngdbf_last_error().decode()


def ngdbf_code_create(n: int, m: int, row_ptr, col_idx) -> int:
    lib = load()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(lib, lib.ngdbf_code_create(n, m, rp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                      ci.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.byref(h)))
    return h.value


def ngdbf_code_destroy(code: int) -> None:
    lib = load()
    _check(lib, lib.ngdbf_code_destroy(code))


def ngdbf_code_info(code: int):
    lib = load()
    v = [ctypes.c_int32() for _ in range(4)]
    _check(lib, lib.ngdbf_code_info(code, *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def ngdbf_decode(code: int, y_ptr: int, n_frames: int, sigma: float, params: ngdbf_params, seed: int,
                 frame_offset: int, bits_ptr: int, iters_ptr: int, pass_ptr: int, stream: int = 0) -> None:
    lib = load()
    _check(lib, lib.ngdbf_decode(code, y_ptr, n_frames, sigma, ctypes.byref(params), seed, frame_offset,
                                 bits_ptr, iters_ptr, pass_ptr, stream))


def ngdbf_decode_plain(code: int, y_ptr: int, n_frames: int, sigma: float, params: ngdbf_params, seed: int,
                       frame_offset: int, bits_ptr: int, iters_ptr: int, pass_ptr: int, stream: int = 0) -> None:
    lib = load()
    _check(lib, lib.ngdbf_decode_plain(code, y_ptr, n_frames, sigma, ctypes.byref(params), seed, frame_offset,
                                       bits_ptr, iters_ptr, pass_ptr, stream))


def ngdbf_decode_trace(code: int, y_ptr: int, n_frames: int, sigma: float, params: ngdbf_params, seed: int,
                       frame_offset: int, bits_ptr: int, iters_ptr: int, pass_ptr: int, trace_frames: int,
                       unsat_ptr: int, corr_ptr: int, stream: int = 0) -> None:
    lib = load()
    _check(lib, lib.ngdbf_decode_trace(code, y_ptr, n_frames, sigma, ctypes.byref(params), seed, frame_offset,
                                       bits_ptr, iters_ptr, pass_ptr, trace_frames, unsat_ptr, corr_ptr, stream))


def ngdbf_decode_noalloc(code: int, y_ptr: int, n_frames: int, sigma: float, params: ngdbf_params,
                         seed: int, frame_offset: int, bits_ptr: int, iters_ptr: int, pass_ptr: int,
                         stream: int = 0) -> None:
    """ngdbf_decode without device allocation: scratch is the library's static device array
    (calls must not overlap on the GPU; the first call on a device should precede any capture)."""
    lib = load()
    _check(lib, lib.ngdbf_decode_noalloc(code, y_ptr, n_frames, sigma, ctypes.byref(params), seed,
                                         frame_offset, bits_ptr, iters_ptr, pass_ptr, stream))


def ngdbf_decode_host(code: int, y_ptr: int, n_frames: int, sigma: float, params: ngdbf_params, seed: int,
                      frame_offset: int, bits_ptr: int, iters_ptr: int, pass_ptr: int,
                      chunk_frames: int = 0) -> None:
    lib = load()
    _check(lib, lib.ngdbf_decode_host(code, y_ptr, n_frames, sigma, ctypes.byref(params), seed,
                                      frame_offset, bits_ptr, iters_ptr, pass_ptr, chunk_frames))


def ngdbf_batch_create(jobs, seed: int, flags: int = 0, stream: int = 0) -> int:
    """jobs: a sequence of ngdbf_job; returns the batch handle."""
    lib = load()
    arr = (ngdbf_job * len(jobs))(*jobs)
    h = ctypes.c_void_p()
    _check(lib, lib.ngdbf_batch_create(arr, len(jobs), seed, flags, stream, ctypes.byref(h)))
    return h.value


def ngdbf_batch_launch(batch: int, stream: int = 0) -> None:
    lib = load()
    _check(lib, lib.ngdbf_batch_launch(batch, stream))


def ngdbf_batch_shape(batch: int, k: int = -1) -> tuple[int, dict]:
    """(number of candidate shapes, description of candidate k; k < 0: the shape in use)."""
    lib = load()
    cnt = ctypes.c_int32()
    info = ngdbf_launch_info()
    _check(lib, lib.ngdbf_batch_shape(batch, k, ctypes.byref(cnt), ctypes.byref(info)))
    return cnt.value, {f: getattr(info, f) for f, _ in info._fields_}


def ngdbf_batch_use_shape(batch: int, k: int) -> None:
    lib = load()
    _check(lib, lib.ngdbf_batch_use_shape(batch, k))


def ngdbf_batch_destroy(batch: int) -> None:
    lib = load()
    _check(lib, lib.ngdbf_batch_destroy(batch))


def ngdbf_server_create(budget_bytes: int, max_inflight: int = 4, max_jobs: int = 256, seed: int = 1) -> int:
    lib = load()
    h = ctypes.c_void_p()
    _check(lib, lib.ngdbf_server_create(budget_bytes, max_inflight, max_jobs, seed, ctypes.byref(h)))
    return h.value


def ngdbf_server_submit(server: int, code: int, y_ptr: int, n_frames: int, sigma: float, params: ngdbf_params,
                        frame_offset: int, bits_ptr: int, iters_ptr: int, pass_ptr: int) -> int:
    lib = load()
    rid = ctypes.c_uint64()
    _check(lib, lib.ngdbf_server_submit(server, code, y_ptr, n_frames, sigma, ctypes.byref(params), frame_offset,
                                        bits_ptr, iters_ptr, pass_ptr, ctypes.byref(rid)))
    return rid.value


def ngdbf_server_poll(server: int, capacity: int = 4096):
    lib = load()
    ids = (ctypes.c_uint64 * capacity)()
    lat = (ctypes.c_double * capacity)()
    st = (ctypes.c_int32 * capacity)()
    n = ctypes.c_int32()
    _check(lib, lib.ngdbf_server_poll(server, ids, lat, st, capacity, ctypes.byref(n)))
    return [(ids[i], lat[i], st[i]) for i in range(n.value)]


def ngdbf_server_wait(server: int, timeout_s: float) -> None:
    lib = load()
    _check(lib, lib.ngdbf_server_wait(server, timeout_s))


def ngdbf_server_get_stats(server: int) -> dict:
    lib = load()
    st = ngdbf_server_stats()
    _check(lib, lib.ngdbf_server_get_stats(server, ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in st._fields_}


def ngdbf_server_destroy(server: int) -> None:
    lib = load()
    _check(lib, lib.ngdbf_server_destroy(server))


def ngdbf_gaussian_range(start: int, count: int, z_ptr: int, stream: int = 0) -> None:
    lib = load()
    _check(lib, lib.ngdbf_gaussian_range(start & 0xFFFFFFFF, count, z_ptr, stream))


def ngdbf_generator_table() -> np.ndarray:
    """[32, 8, 4] FP32 coefficients of the generator's inverse-CDF segments (host call)."""
    lib = load()
    out = np.empty((32, 8, 4), dtype=np.float32)
    _check(lib, lib.ngdbf_generator_table(out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    return out


def ngdbf_mix_probe(groups: int, sink_ptr: int, stream: int = 0) -> int:
    """Launches the same-mix throughput probe; returns the number of threads launched."""
    lib = load()
    th = ctypes.c_int64()
    _check(lib, lib.ngdbf_mix_probe(groups, sink_ptr, ctypes.byref(th), stream))
    return th.value


def ngdbf_pool_usage(reset_high: bool = False) -> tuple[int, int]:
    """(bytes in use now, most bytes in use since the last reset) of the library's scratch pool."""
    lib = load()
    now, high = ctypes.c_int64(), ctypes.c_int64()
    _check(lib, lib.ngdbf_pool_usage(1 if reset_high else 0, ctypes.byref(now), ctypes.byref(high)))
    return now.value, high.value


def ngdbf_host_alloc(nbytes: int) -> int:
    """Page-locked host block of nbytes (huge-page backed when large); free with ngdbf_host_free."""
    lib = load()
    p = ctypes.c_void_p()
    _check(lib, lib.ngdbf_host_alloc(nbytes, ctypes.byref(p)))
    return p.value


def ngdbf_host_free(ptr: int) -> None:
    lib = load()
    _check(lib, lib.ngdbf_host_free(ptr))


def ngdbf_host_huge_page_bytes() -> int:
    lib = load()
    v = ctypes.c_int64()
    _check(lib, lib.ngdbf_host_huge_page_bytes(ctypes.byref(v)))
    return v.value


def ngdbf_host_block_info(ptr: int) -> tuple[int, int]:
    """(mapped bytes, bytes backed by huge pages) of a block from ngdbf_host_alloc."""
    lib = load()
    b, h = ctypes.c_int64(), ctypes.c_int64()
    _check(lib, lib.ngdbf_host_block_info(ptr, ctypes.byref(b), ctypes.byref(h)))
    return b.value, h.value


NGDBF_HOST_COPY_STAGED = 0
NGDBF_HOST_COPY_DIRECT = 1


def ngdbf_set_host_copy_mode(mode: int) -> None:
    lib = load()
    _check(lib, lib.ngdbf_set_host_copy_mode(mode))


def ngdbf_get_host_copy_mode() -> int:
    lib = load()
    v = ctypes.c_int32()
    _check(lib, lib.ngdbf_get_host_copy_mode(ctypes.byref(v)))
    return v.value


def host_empty(shape, dtype=np.float32):
    """A CPU torch tensor over a block from ngdbf_host_alloc (page-locked; returned to the
    library when the tensor and its views are gone)."""
    import weakref
    import torch
    shape = tuple(int(d) for d in (shape if isinstance(shape, (tuple, list)) else (shape,)))
    dt = np.dtype(dtype)
    nbytes = max(1, int(np.prod(shape, dtype=np.int64)) * dt.itemsize)
    ptr = ngdbf_host_alloc(nbytes)
    raw = (ctypes.c_uint8 * nbytes).from_address(ptr)
    weakref.finalize(raw, ngdbf_host_free, ptr)
    arr = np.frombuffer(raw, dtype=np.uint8, count=nbytes)
    arr = arr[: int(np.prod(shape, dtype=np.int64)) * dt.itemsize].view(dt).reshape(shape)
    return torch.from_numpy(arr)


def ngdbf_last_host_stats() -> dict:
    """Event timing of the calling thread's most recent ngdbf_decode_host (ms, bytes)."""
    lib = load()
    st = ngdbf_host_stats()
    _check(lib, lib.ngdbf_last_host_stats(ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in st._fields_ if f != "reserved"}


def ngdbf_last_launch() -> dict:
    lib = load()
    info = ngdbf_launch_info()
    _check(lib, lib.ngdbf_last_launch(ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in info._fields_}


# --- convenience over torch device memory -----------------------------------------------------------

class DeviceCode:
    """A parity-check matrix resident on the current CUDA device."""

    def __init__(self, n: int, m: int, row_ptr, col_idx):
        self.n, self.m = int(n), int(m)
        self.handle = ngdbf_code_create(self.n, self.m, row_ptr, col_idx)

    @classmethod
    def from_code(cls, code) -> "DeviceCode":
        return cls(code.n, code.m, code.row_ptr, code.col_idx)

    def close(self) -> None:
        if self.handle:
            ngdbf_code_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def decode(self, y, sigma: float, params: ngdbf_params, seed: int = 1, frame_offset: int = 0,
               out=None, stream=None):
        """y: float32 CUDA tensor [F, n].  Returns (bits uint8 [F, ceil(n/8)], iters int32 [F],
        pass uint8 [F]) as CUDA tensors, enqueued on ``stream`` (default: torch's current stream)."""
        import torch
        assert y.is_cuda and y.dtype == torch.float32 and y.is_contiguous() and y.shape[-1] == self.n
        F = y.shape[0]
        if out is None:
            bits = torch.empty((F, (self.n + 7) // 8), dtype=torch.uint8, device=y.device)
            iters = torch.empty(F, dtype=torch.int32, device=y.device)
            pas = torch.empty(F, dtype=torch.uint8, device=y.device)
        else:
            bits, iters, pas = out
        s = stream if stream is not None else torch.cuda.current_stream(y.device)
        ngdbf_decode(self.handle, y.data_ptr(), F, float(sigma), params, int(seed), int(frame_offset),
                     bits.data_ptr(), iters.data_ptr(), pas.data_ptr(), s.cuda_stream)
        return bits, iters, pas

    def decode_plain(self, y, sigma: float, params: ngdbf_params, seed: int = 1, frame_offset: int = 0,
                     out=None, stream=None):
        """decode() by the plain per-iteration kernels (baseline form; same results)."""
        import torch
        assert y.is_cuda and y.dtype == torch.float32 and y.is_contiguous() and y.shape[-1] == self.n
        F = y.shape[0]
        if out is None:
            out = (torch.empty((F, (self.n + 7) // 8), dtype=torch.uint8, device=y.device),
                   torch.empty(F, dtype=torch.int32, device=y.device), torch.empty(F, dtype=torch.uint8, device=y.device))
        bits, iters, pas = out
        s = stream if stream is not None else torch.cuda.current_stream(y.device)
        ngdbf_decode_plain(self.handle, y.data_ptr(), F, float(sigma), params, int(seed), int(frame_offset),
                           bits.data_ptr(), iters.data_ptr(), pas.data_ptr(), s.cuda_stream)
        return bits, iters, pas

    def decode_trace(self, y, sigma: float, params: ngdbf_params, trace_frames: int, seed: int = 1,
                     frame_offset: int = 0, stream=None):
        """decode() plus the objective trace of the first trace_frames frames: returns (bits, iters,
        pass, U int32 [K, T+1], C int64 [K, T+1]) as CUDA tensors; U is -1 and C 0 after iters[f]."""
        import torch
        assert y.is_cuda and y.dtype == torch.float32 and y.is_contiguous() and y.shape[-1] == self.n
        F, K, T = y.shape[0], int(trace_frames), params.t_max
        bits = torch.empty((F, (self.n + 7) // 8), dtype=torch.uint8, device=y.device)
        iters = torch.empty(F, dtype=torch.int32, device=y.device)
        pas = torch.empty(F, dtype=torch.uint8, device=y.device)
        tu = torch.full((max(K, 1), T + 1), -1, dtype=torch.int32, device=y.device)
        tc = torch.zeros((max(K, 1), T + 1), dtype=torch.int64, device=y.device)
        s = stream if stream is not None else torch.cuda.current_stream(y.device)
        ngdbf_decode_trace(self.handle, y.data_ptr(), F, float(sigma), params, int(seed), int(frame_offset),
                           bits.data_ptr(), iters.data_ptr(), pas.data_ptr(), K, tu.data_ptr(), tc.data_ptr(),
                           s.cuda_stream)
        return bits, iters, pas, tu[:K], tc[:K]

    def decode_host(self, y: np.ndarray, sigma: float, params: ngdbf_params, seed: int = 1,
                    frame_offset: int = 0, out=None, chunk_frames: int = 0):
        """Host arrays in and out (numpy or pinned CPU torch tensors)."""
        F = y.shape[0]
        if out is None:
            bits = np.empty((F, (self.n + 7) // 8), dtype=np.uint8)
            iters = np.empty(F, dtype=np.int32)
            pas = np.empty(F, dtype=np.uint8)
        else:
            bits, iters, pas = out

        def ptr(a):
            return a.ctypes.data if isinstance(a, np.ndarray) else a.data_ptr()
        ngdbf_decode_host(self.handle, ptr(y), F, float(sigma), params, int(seed), int(frame_offset),
                          ptr(bits), ptr(iters), ptr(pas), chunk_frames)
        return bits, iters, pas


class Batch:
    """Several decode jobs (DeviceCode, CUDA samples, sigma, params, frame offset) in one launch;
    outputs are allocated here as CUDA tensors (bits, iters, pass per job)."""

    def __init__(self, jobs, seed: int = 1, flags: int = NGDBF_BATCH_GRAPH, stream=None):
        import torch
        self.outputs, cj = [], []
        for code, y, sigma, params, frame_offset in jobs:
            F = y.shape[0]
            bits = torch.empty((F, (code.n + 7) // 8), dtype=torch.uint8, device=y.device)
            iters = torch.empty(F, dtype=torch.int32, device=y.device)
            pas = torch.empty(F, dtype=torch.uint8, device=y.device)
            self.outputs.append((bits, iters, pas))
            cj.append(ngdbf_job(code.handle, y.data_ptr(), F, float(sigma), params, int(frame_offset),
                                bits.data_ptr(), iters.data_ptr(), pas.data_ptr()))
        self._keep = [j for j in jobs]
        s = stream if stream is not None else torch.cuda.current_stream()
        self.handle = ngdbf_batch_create(cj, seed, flags, s.cuda_stream)

    def launch(self, stream=None):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        ngdbf_batch_launch(self.handle, s.cuda_stream)
        return self.outputs

    def shapes(self) -> list[dict]:
        """The candidate launch shapes (block, cluster, placement, ...)."""
        n, _ = ngdbf_batch_shape(self.handle, 0)
        return [ngdbf_batch_shape(self.handle, k)[1] for k in range(n)]

    def shape(self) -> dict:
        return ngdbf_batch_shape(self.handle, -1)[1]

    def use_shape(self, k: int) -> None:
        ngdbf_batch_use_shape(self.handle, k)

    def close(self):
        if self.handle:
            ngdbf_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching decode server over host buffers (numpy arrays or pinned CPU tensors)."""

    def __init__(self, budget_bytes: int, max_inflight: int = 4, max_jobs: int = 256, seed: int = 1):
        self.handle = ngdbf_server_create(budget_bytes, max_inflight, max_jobs, seed)
        self._live = {}

    @staticmethod
    def _ptr(a):
        return a.ctypes.data if isinstance(a, np.ndarray) else a.data_ptr()

    def submit(self, code: "DeviceCode", y, sigma: float, params: ngdbf_params, frame_offset: int = 0, out=None):
        F = y.shape[0]
        if out is None:
            out = (np.empty((F, (code.n + 7) // 8), np.uint8), np.empty(F, np.int32), np.empty(F, np.uint8))
        rid = ngdbf_server_submit(self.handle, code.handle, self._ptr(y), F, float(sigma), params,
                                  int(frame_offset), *[self._ptr(o) for o in out])
        self._live[rid] = (y, out, code)          # keep buffers alive until completion
        return rid, out

    def poll(self):
        done = ngdbf_server_poll(self.handle)
        for rid, _, _ in done:
            self._live.pop(rid, None)
        return done

    def wait(self, timeout_s: float = 600.0):
        ngdbf_server_wait(self.handle, timeout_s)

    def stats(self) -> dict:
        return ngdbf_server_get_stats(self.handle)

    def close(self):
        if self.handle:
            ngdbf_server_destroy(self.handle)
            self.handle = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
