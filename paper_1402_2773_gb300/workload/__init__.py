"""Seeded synthetic LDPC workloads: codes, codewords and AWGN frames.

This module produces the inputs that the decoder library and the reference
(oracle) decoder both consume.  It holds none of the decoder's arithmetic.

* ``peg_code(n, m, dv, seed)`` builds a parity-check matrix by progressive
  edge growth (Hu, Eleftheriou, Arnold 2005) with symbol degree ``dv`` and
  balanced check degrees; it stands in for the MacKay codes the paper
  simulates (Sec. IV-A), which are not available here.
* ``Code.encoder()`` runs Gaussian elimination over GF(2) to a reduced
  row-echelon form; the non-pivot columns are the information positions and
  every pivot row gives one parity bit (a systematic encoder).
* ``frames(code, F, ebn0_db, seed)`` draws information words, encodes them,
  maps c -> 1 - 2c (paper Sec. III-A) and adds Gaussian noise with
  variance N0/2 = 1 / (2 R Eb/N0) (the reading of Sec. III-A/IV-A used
  throughout; it gives sigma = 0.668 at 3.5 dB for R = 1/2, Sec. VII).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "workload.c")
_LIB_PATH = os.path.join(_HERE, "libngdbf_workload.so")
_lib = None


def build(force: bool = False) -> str:
    """Compiles the workload helper library with gcc (host code only)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = f"{_LIB_PATH}.{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-D_GNU_SOURCE",
                               "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.wl_peg.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, i32p, i32p]
        lib.wl_peg.restype = ctypes.c_int
        lib.wl_frames.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, i32p, i32p,
                                  ctypes.POINTER(ctypes.c_uint64), ctypes.c_int64, ctypes.c_double,
                                  ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int32,
                                  ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_uint8)]
        lib.wl_frames.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


@dataclass
class Encoder:
    """Systematic GF(2) encoder: parity bit p = popcount(pmask[p] & info) mod 2."""
    rank: int
    info_pos: np.ndarray      # int32 [k]
    pivot_pos: np.ndarray     # int32 [rank]
    pmask: np.ndarray         # uint64 [rank][ceil(k/64)]

    @property
    def k(self) -> int:
        return int(self.info_pos.size)


@dataclass
class Code:
    """Parity-check matrix H (m x n) in CSR form: row i lists N(i)."""
    n: int
    m: int
    row_ptr: np.ndarray       # int32 [m+1]
    col_idx: np.ndarray       # int32 [nnz]
    name: str = ""
    _enc: Encoder | None = field(default=None, repr=False)

    def dense(self) -> np.ndarray:
        H = np.zeros((self.m, self.n), dtype=np.uint8)
        rows = np.repeat(np.arange(self.m), np.diff(self.row_ptr))
        H[rows, self.col_idx] = 1
        return H

    def encoder(self) -> Encoder:
        if self._enc is None:
            self._enc = _gf2_encoder(self.dense())
        return self._enc

    @property
    def rank(self) -> int:
        return self.encoder().rank

    @property
    def k(self) -> int:
        return self.n - self.rank

    @property
    def rate(self) -> float:
        return self.k / self.n


def _gf2_encoder(H: np.ndarray) -> Encoder:
    """Reduced row-echelon form of H over GF(2), pivots chosen left to right."""
    m, n = H.shape
    A = H.astype(bool).copy()
    pivots = []
    row = 0
    for col in range(n):
        if row >= m:
            break
        nz = np.nonzero(A[row:, col])[0]
        if nz.size == 0:
            continue
        p = row + int(nz[0])
        if p != row:
            A[[row, p]] = A[[p, row]]
        others = np.nonzero(A[:, col])[0]
        others = others[others != row]
        if others.size:
            A[others] ^= A[row]
        pivots.append(col)
        row += 1
    r = len(pivots)
    piv = np.array(pivots, dtype=np.int32)
    is_piv = np.zeros(n, dtype=bool)
    is_piv[piv] = True
    info = np.nonzero(~is_piv)[0].astype(np.int32)
    k = info.size
    kw = max(1, (k + 63) // 64)
    # Row i of the RREF reads c[piv[i]] + sum_{j in info} A[i, j] c[j] = 0.
    sub = A[:r][:, info]
    padded = np.zeros((r, kw * 64), dtype=np.uint8)
    padded[:, :k] = sub
    pm = np.packbits(padded, axis=1, bitorder="little").view("<u8").reshape(r, kw)
    return Encoder(rank=r, info_pos=info, pivot_pos=piv, pmask=np.ascontiguousarray(pm, dtype=np.uint64))


def peg_code(n: int, m: int, dv: int, seed: int = 1, name: str = "") -> Code:
    """Progressive-edge-growth code with symbol degree dv and balanced check degrees."""
    lib = _load()
    nnz = n * dv
    row_ptr = np.zeros(m + 1, dtype=np.int32)
    col_idx = np.zeros(nnz, dtype=np.int32)
    rc = lib.wl_peg(n, m, dv, seed, _ptr(row_ptr, ctypes.c_int32), _ptr(col_idx, ctypes.c_int32))
    if rc != 0:
        raise RuntimeError(f"wl_peg failed ({rc}) for n={n} m={m} dv={dv}")
    return Code(n=n, m=m, row_ptr=row_ptr, col_idx=col_idx, name=name or f"peg_{dv}_{n}x{m}_s{seed}")


def code_from_dense(H: np.ndarray, name: str = "") -> Code:
    H = np.asarray(H, dtype=np.uint8)
    m, n = H.shape
    row_ptr = np.zeros(m + 1, dtype=np.int32)
    cols = []
    for i in range(m):
        c = np.nonzero(H[i])[0]
        cols.append(c)
        row_ptr[i + 1] = row_ptr[i] + c.size
    col_idx = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32)
    return Code(n=n, m=m, row_ptr=row_ptr, col_idx=col_idx, name=name or f"dense_{n}x{m}")


def sigma_for(ebn0_db: float, rate: float) -> float:
    """Channel noise std for BPSK at Eb/N0 (dB): sigma^2 = N0/2 = 1 / (2 R Eb/N0)."""
    return math.sqrt(1.0 / (2.0 * rate * 10.0 ** (ebn0_db / 10.0)))


def frames(code: Code, n_frames: int, ebn0_db: float | None, seed: int = 1, frame_offset: int = 0,
           threads: int | None = None, sigma: float | None = None, out: np.ndarray | None = None):
    """Draws n_frames AWGN frames.

    Returns (y float32 [F, n], codeword bits uint8 [F, ceil(n/8)] LSB-first,
    sigma).  ``ebn0_db=None`` with ``sigma=None`` gives noiseless frames.
    ``out`` may supply a preallocated (e.g. pinned) float32 [F, n] buffer.
    """
    lib = _load()
    enc = code.encoder()
    if sigma is None:
        sigma = -1.0 if ebn0_db is None else sigma_for(ebn0_db, code.rate)
    if out is None:
        y = np.empty((n_frames, code.n), dtype=np.float32)
    else:
        y = out
        assert y.dtype == np.float32 and y.shape == (n_frames, code.n) and y.flags.c_contiguous
    cw = np.empty((n_frames, (code.n + 7) // 8), dtype=np.uint8)
    if threads is None:
        threads = os.cpu_count() or 1
    rc = lib.wl_frames(code.n, enc.k, enc.rank, _ptr(enc.info_pos, ctypes.c_int32),
                       _ptr(enc.pivot_pos, ctypes.c_int32), _ptr(enc.pmask, ctypes.c_uint64),
                       n_frames, float(sigma), seed, frame_offset, threads,
                       _ptr(y, ctypes.c_float), _ptr(cw, ctypes.c_uint8))
    if rc != 0:
        raise RuntimeError("wl_frames failed")
    return y, cw, (sigma if sigma >= 0 else 0.0)


def unpack_bits(packed: np.ndarray, n: int) -> np.ndarray:
    """[F, ceil(n/8)] LSB-first bytes -> [F, n] uint8 bits."""
    return np.unpackbits(packed, axis=-1, count=n, bitorder="little")


# Workload shapes of the paper's experiments (Sec. IV), as seeded PEG stand-ins.
def code_c1(seed: int = 1) -> Code:
    """(3,6)-regular, N=1008, M=504: the shape of PEGReg504x1008 (Sec. IV-A)."""
    return peg_code(1008, 504, 3, seed, name="peg(3,6) N=1008 M=504")


def code_c2(seed: int = 1) -> Code:
    """(6,32)-regular, N=2048, M=384: a high-rate code (cf. the (4,62) code of Fig. 5)."""
    return peg_code(2048, 384, 6, seed, name="peg(6,32) N=2048 M=384")
