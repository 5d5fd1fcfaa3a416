"""Reference (oracle) NGDBF decoder -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``ngdbf_oracle.c`` (plain C,
no FMA contraction, strict IEEE FP32/FP64) through ctypes and shares no code
with the CUDA decoder in ``paper_1402_2773_gb300``.

Functions follow the paper (Sundararajan, Winstead, Boutillon 2014):
``decode_f32`` / ``decode_f64`` run Steps 0-3b of Sec. III-B/C/D with the
smoothing of Sec. III-E; ``quantize`` is g(.) of Sec. IV-E (Eq. 8);
``threshold_events`` is the (theta~, tau~) list of Sec. V-A (Table II).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(_HERE, "ngdbf_oracle.c")
LIB_PATH = os.path.join(_HERE, "libngdbf_oracle.so")
CFLAGS = ["-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
          "-D_GNU_SOURCE"]

ADAPT = 1
SMOOTH = 2
SINGLE = 4
UNIFORM = 8
FP32 = 0
FP16 = 1
FIX = 2
FIXACC = 3
ACC_BITS = 8


class Params(ctypes.Structure):
    _fields_ = [("w", ctypes.c_float), ("theta", ctypes.c_float), ("eta", ctypes.c_float),
                ("lambda_", ctypes.c_float), ("y_max", ctypes.c_float),
                ("t_max", ctypes.c_int32), ("smooth_window", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("q_bits", ctypes.c_int32)]


def make_params(w=0.75, theta=-0.9, eta=0.96, lam=1.0, y_max=2.5, t_max=100, smooth_window=64,
                variant=0, precision=0, q_bits=8) -> Params:
    return Params(w, theta, eta, lam, y_max, t_max, smooth_window, variant, precision, q_bits)


def compile_lib(src: str = SRC, out: str = LIB_PATH, extra: list[str] | None = None) -> str:
    """Compiles an oracle source file into a shared library (gcc)."""
    tmp = f"{out}.{os.getpid()}.tmp"
    subprocess.check_call(["gcc", *CFLAGS, *(extra or []), "-o", tmp, src, "-lm", "-lpthread"])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < os.path.getmtime(SRC):
        compile_lib()
    return LIB_PATH


class Oracle:
    """ctypes view of one compiled oracle library (the default one or a test build)."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        i32p = ctypes.POINTER(ctypes.c_int32)
        f32p = ctypes.POINTER(ctypes.c_float)
        f64p = ctypes.POINTER(ctypes.c_double)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        lib.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
        lib.oracle_philox4x32_10.restype = None
        lib.oracle_gauss_f32.argtypes = [ctypes.c_uint32]
        lib.oracle_gauss_f32.restype = ctypes.c_float
        lib.oracle_gauss_f64.argtypes = [ctypes.c_uint32]
        lib.oracle_gauss_f64.restype = ctypes.c_double
        lib.oracle_gauss_range_f32.argtypes = [ctypes.c_uint32, ctypes.c_uint32, f32p]
        lib.oracle_gauss_range_f32.restype = None
        lib.oracle_gauss_many_f32.argtypes = [u32p, ctypes.c_uint32, f32p]
        lib.oracle_gauss_many_f32.restype = None
        lib.oracle_icdf_table.argtypes = [f32p]
        lib.oracle_icdf_table.restype = None
        for nm, zt in (("oracle_gauss4_f32", f32p), ("oracle_gauss4_f64", f64p)):
            fn = getattr(lib, nm)
            fn.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, zt]
            fn.restype = None
        lib.oracle_uniform_f32.argtypes = [ctypes.c_uint32]
        lib.oracle_uniform_f32.restype = ctypes.c_float
        lib.oracle_uniform4_f32.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, f32p]
        lib.oracle_uniform4_f32.restype = None
        lib.oracle_fixacc_scale.argtypes = [ctypes.c_int32, ctypes.c_float]
        lib.oracle_fixacc_scale.restype = ctypes.c_float
        lib.oracle_fixacc_steps.argtypes = [ctypes.c_float, ctypes.c_float]
        lib.oracle_fixacc_steps.restype = ctypes.c_int32
        lib.oracle_noise_f32.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                         ctypes.c_float, ctypes.c_float]
        lib.oracle_noise_f32.restype = ctypes.c_float
        lib.oracle_threshold_table_f32.argtypes = [ctypes.c_float, ctypes.c_float, ctypes.c_int32, f32p]
        lib.oracle_threshold_table_f32.restype = None
        lib.oracle_metric_f32.argtypes = [ctypes.c_int, ctypes.c_float, ctypes.c_int, ctypes.c_float,
                                          ctypes.c_float]
        lib.oracle_metric_f32.restype = ctypes.c_float
        lib.oracle_metric_f16.argtypes = [ctypes.c_int, ctypes.c_float, ctypes.c_int, ctypes.c_float,
                                          ctypes.c_float]
        lib.oracle_metric_f16.restype = ctypes.c_float
        lib.oracle_metric_f64.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                          ctypes.c_double]
        lib.oracle_metric_f64.restype = ctypes.c_double
        lib.oracle_quantize.argtypes = [ctypes.c_double, ctypes.c_int32, ctypes.c_double]
        lib.oracle_quantize.restype = ctypes.c_double
        lib.oracle_round_half.argtypes = [ctypes.c_float]
        lib.oracle_round_half.restype = ctypes.c_float
        lib.oracle_fix_scale.argtypes = [ctypes.c_int32, ctypes.c_float]
        lib.oracle_fix_scale.restype = ctypes.c_float
        lib.oracle_fix_code.argtypes = [ctypes.c_float, ctypes.c_float, ctypes.c_int32]
        lib.oracle_fix_code.restype = ctypes.c_int32
        lib.oracle_threshold_events.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                                ctypes.c_int32, ctypes.c_double, f64p, i32p,
                                                ctypes.c_int32]
        lib.oracle_threshold_events.restype = ctypes.c_int32
        dec = [ctypes.c_int32, ctypes.c_int32, i32p, i32p, f32p, ctypes.c_int64, ctypes.c_float,
               ctypes.POINTER(Params), ctypes.c_uint64, ctypes.c_uint64, u8p, i32p, u8p, ctypes.c_int32]
        for nm in ("oracle_decode_f32", "oracle_decode_f64"):
            fn = getattr(lib, nm)
            fn.argtypes = dec
            fn.restype = ctypes.c_int
        i64p = ctypes.POINTER(ctypes.c_int64)
        for nm in ("oracle_decode_f32_trace", "oracle_decode_f64_trace"):
            fn = getattr(lib, nm)
            fn.argtypes = dec + [ctypes.c_int64, i32p, i64p]
            fn.restype = ctypes.c_int
        lib.oracle_decode_f32_qin.argtypes = [ctypes.c_int32, ctypes.c_int32, i32p, i32p, f32p,
                                              ctypes.POINTER(Params), f32p, u8p, i32p, u8p]
        lib.oracle_decode_f32_qin.restype = ctypes.c_int
        self.lib = lib

    # -- generator -----------------------------------------------------------
    def philox(self, ctr, key) -> np.ndarray:
        c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
        k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
        o = (ctypes.c_uint32 * 4)()
        self.lib.oracle_philox4x32_10(c, k, o)
        return np.array(list(o), dtype=np.uint32)

    def gauss_f32(self, r: int) -> np.float32:
        """FP32 standard normal deviate of one Philox output r (inverse normal CDF)."""
        return np.float32(self.lib.oracle_gauss_f32(ctypes.c_uint32(int(r) & 0xFFFFFFFF)))

    def gauss_f64(self, r: int) -> float:
        return float(self.lib.oracle_gauss_f64(ctypes.c_uint32(int(r) & 0xFFFFFFFF)))

    def gauss_range_f32(self, start: int, count: int) -> np.ndarray:
        """Deviates of r = start .. start + count - 1."""
        out = np.empty(count, dtype=np.float32)
        self.lib.oracle_gauss_range_f32(start, count, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
        return out

    def gauss_many_f32(self, r) -> np.ndarray:
        """Deviates of the outputs in the array r."""
        r = np.ascontiguousarray(r, dtype=np.uint32)
        out = np.empty(r.shape[0], dtype=np.float32)
        self.lib.oracle_gauss_many_f32(r.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), r.shape[0],
                                       out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
        return out

    def icdf_table(self) -> np.ndarray:
        """[32, 8, 4] FP32 cubic coefficients, segment (level j, sub-interval s)."""
        out = np.empty((32, 8, 4), dtype=np.float32)
        self.lib.oracle_icdf_table(out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
        return out

    def gauss4_f32(self, seed, frame, t, g) -> np.ndarray:
        z = (ctypes.c_float * 4)()
        self.lib.oracle_gauss4_f32(seed, frame, t, g, z)
        return np.array(list(z), dtype=np.float32)

    def gauss4_f64(self, seed, frame, t, g) -> np.ndarray:
        z = (ctypes.c_double * 4)()
        self.lib.oracle_gauss4_f64(seed, frame, t, g, z)
        return np.array(list(z), dtype=np.float64)

    def uniform_f32(self, r: int) -> np.float32:
        """Uniform deviate on (-1, 1) of one Philox output r (Sec. V-B variant)."""
        return np.float32(self.lib.oracle_uniform_f32(ctypes.c_uint32(int(r) & 0xFFFFFFFF)))

    def uniform4_f32(self, seed, frame, t, g) -> np.ndarray:
        v = (ctypes.c_float * 4)()
        self.lib.oracle_uniform4_f32(seed, frame, t, g, v)
        return np.array(list(v), dtype=np.float32)

    def fixacc_scale(self, q_bits: int, y_max: float) -> float:
        """Rd = fl32(2^(Q+8) / Y_max), accumulator steps per unit of the FIXACC form."""
        return float(np.float32(self.lib.oracle_fixacc_scale(q_bits, y_max)))

    def fixacc_steps(self, v: float, Rd: float) -> int:
        return int(self.lib.oracle_fixacc_steps(v, Rd))

    def noise_f32(self, seed, frame, t, k, eta, sigma) -> np.float32:
        return np.float32(self.lib.oracle_noise_f32(seed, frame, t, k, eta, sigma))

    # -- thresholds / metric / quantizer ---------------------------------------
    def threshold_table_f32(self, theta, lam, t_max) -> np.ndarray:
        out = np.empty(t_max + 1, dtype=np.float32)
        self.lib.oracle_threshold_table_f32(theta, lam, t_max, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
        return out

    def metric_f32(self, x: int, ys: float, S: int, w: float, q: float) -> np.float32:
        return np.float32(self.lib.oracle_metric_f32(x, ys, S, w, q))

    def metric_f16(self, x: int, ys16: float, S: int, w16: float, q: float) -> float:
        return float(np.float32(self.lib.oracle_metric_f16(x, ys16, S, w16, q)))

    def metric_f64(self, x: int, ys: float, S: int, w: float, q: float) -> float:
        return float(self.lib.oracle_metric_f64(x, ys, S, w, q))

    def quantize(self, v: float, q_bits: int, y_max: float) -> float:
        return float(self.lib.oracle_quantize(v, q_bits, y_max))

    def round_half(self, x: float) -> float:
        return float(np.float32(self.lib.oracle_round_half(ctypes.c_float(x))))

    def fix_scale(self, q_bits: int, y_max: float) -> float:
        return float(np.float32(self.lib.oracle_fix_scale(q_bits, y_max)))

    def fix_code(self, v: float, R: float, kmax: int) -> int:
        return int(self.lib.oracle_fix_code(v, R, kmax))

    def threshold_events(self, theta, lam, t_max, q_bits, y_max, cap=64):
        thr = np.zeros(cap, dtype=np.float64)
        tau = np.zeros(cap, dtype=np.int32)
        cnt = self.lib.oracle_threshold_events(theta, lam, t_max, q_bits, y_max,
                                               thr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                               tau.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), cap)
        return list(zip(thr[:cnt].tolist(), tau[:cnt].tolist()))

    # -- decoders ----------------------------------------------------------------
    def _decode(self, fn, code, y, sigma, params, seed, frame_offset, threads, trace=None):
        y = np.ascontiguousarray(y, dtype=np.float32)
        F = y.shape[0]
        nb = (code.n + 7) // 8
        bits = np.zeros((F, nb), dtype=np.uint8)
        iters = np.zeros(F, dtype=np.int32)
        pas = np.zeros(F, dtype=np.uint8)
        rp = np.ascontiguousarray(code.row_ptr, dtype=np.int32)
        ci = np.ascontiguousarray(code.col_idx, dtype=np.int32)
        args = [code.n, code.m, rp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                ci.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                y.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), F, sigma, ctypes.byref(params),
                seed, frame_offset, bits.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                iters.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                pas.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), threads]
        if trace is not None:
            tu, tc = trace
            args += [tu.shape[0], tu.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                     tc.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))]
        rc = fn(*args)
        if rc != 0:
            raise RuntimeError(f"oracle decode failed ({rc})")
        return bits, iters, pas

    def _decode_trace(self, fn, code, y, sigma, params, seed, frame_offset, threads, trace_frames):
        K = int(trace_frames)
        tu = np.full((K, params.t_max + 1), -1, dtype=np.int32)
        tc = np.zeros((K, params.t_max + 1), dtype=np.int64)
        bits, iters, pas = self._decode(fn, code, y, sigma, params, seed, frame_offset, threads, (tu, tc))
        return bits, iters, pas, tu, tc

    def decode_f32_trace(self, code, y, sigma, params, trace_frames, seed=1, frame_offset=0, threads=1):
        """FP32 decode with the objective trace of the first trace_frames frames: returns
        (bits, iters, pass, U [K][T+1] int32, C [K][T+1] int64); entries after iters[f] stay -1 / 0.
        f(x(t)) = C 2^-32 + m - 2 U (Sec. III-B objective)."""
        return self._decode_trace(self.lib.oracle_decode_f32_trace, code, y, sigma, params, seed,
                                  frame_offset, threads, trace_frames)

    def decode_f64_trace(self, code, y, sigma, params, trace_frames, seed=1, frame_offset=0, threads=1):
        return self._decode_trace(self.lib.oracle_decode_f64_trace, code, y, sigma, params, seed,
                                  frame_offset, threads, trace_frames)

    def decode_f32(self, code, y, sigma, params, seed=1, frame_offset=0, threads=1):
        return self._decode(self.lib.oracle_decode_f32, code, y, sigma, params, seed, frame_offset, threads)

    def decode_f64(self, code, y, sigma, params, seed=1, frame_offset=0, threads=1):
        return self._decode(self.lib.oracle_decode_f64, code, y, sigma, params, seed, frame_offset, threads)

    def decode_f32_qin(self, code, y, params, q):
        """One frame with given perturbations q[t][k] (t < t_max)."""
        y = np.ascontiguousarray(y, dtype=np.float32).reshape(-1)
        q = np.ascontiguousarray(q, dtype=np.float32)
        assert q.shape == (params.t_max, code.n) or params.t_max == 0
        nb = (code.n + 7) // 8
        bits = np.zeros(nb, dtype=np.uint8)
        it = ctypes.c_int32()
        ps = ctypes.c_uint8()
        rp = np.ascontiguousarray(code.row_ptr, dtype=np.int32)
        ci = np.ascontiguousarray(code.col_idx, dtype=np.int32)
        qq = q if q.size else np.zeros(1, np.float32)
        rc = self.lib.oracle_decode_f32_qin(
            code.n, code.m, rp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
            ci.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
            y.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(params),
            qq.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
            bits.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), ctypes.byref(it), ctypes.byref(ps))
        if rc != 0:
            raise RuntimeError("oracle decode failed")
        return bits, int(it.value), int(ps.value)


_default: Oracle | None = None


def load() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle(build())
    return _default
