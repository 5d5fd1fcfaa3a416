"""Objective function and convergence error of a decode (Sec. III-B Eq. 2, Sec. VI Eqs. 17-18).

f(x) = sum_k x_k y_k + sum_i s_i(x) is the GDBF objective; for a codeword every
s_i = +1, so the transmitted word reaches f_max = sum_k c^_k y_k + m.  The
convergence error of a set of frames is the mean of f(x(T)) - f_max over them,
where x(T) is the decoder's output.  These are host-side evaluations of decode
results (numpy); they are not part of the decode itself.  Samples are taken as
the decoder holds them: saturated to [-y_max, y_max] when y_max > 0.
"""
from __future__ import annotations

import numpy as np


def _held(y: np.ndarray, y_max: float | None) -> np.ndarray:
    y = np.asarray(y, dtype=np.float64)
    if y_max is not None and y_max > 0 and np.isfinite(y_max):
        y = np.clip(y, -y_max, y_max)
    return y


def bipolar(bits: np.ndarray, n: int) -> np.ndarray:
    """[F, ceil(n/8)] packed decisions (bit 1 <=> x = -1) -> [F, n] values in {+1, -1}."""
    b = np.unpackbits(np.asarray(bits, dtype=np.uint8), axis=-1, count=n, bitorder="little")
    return 1.0 - 2.0 * b.astype(np.float64)


def syndrome_sum(code, x: np.ndarray) -> np.ndarray:
    """sum_i s_i with s_i = prod_{j in N(i)} x_j, per frame ([F, n] bipolar -> [F])."""
    neg = (x < 0).astype(np.int64)
    rows = np.repeat(np.arange(code.m), np.diff(code.row_ptr))
    odd = np.zeros((x.shape[0], code.m), dtype=np.int64)
    np.add.at(odd.T, rows, neg[:, code.col_idx].T)
    s = 1 - 2 * (odd % 2)
    return s.sum(axis=1)


def objective(code, y: np.ndarray, bits: np.ndarray, y_max: float | None = None) -> np.ndarray:
    """f(x) of Eq. 2 for each frame's decoded word."""
    x = bipolar(bits, code.n)
    return (x * _held(y, y_max)).sum(axis=1) + syndrome_sum(code, x)


def f_max(code, y: np.ndarray, codewords: np.ndarray, y_max: float | None = None) -> np.ndarray:
    """f of the transmitted codeword: sum_k c^_k y_k + m (Sec. VI)."""
    c = bipolar(codewords, code.n)
    return (c * _held(y, y_max)).sum(axis=1) + code.m


def convergence_error(code, y, bits, codewords, y_max: float | None = None) -> float:
    """epsilon of Eq. 17: mean over frames of f(x(T)) - f_max."""
    return float(np.mean(objective(code, y, bits, y_max) - f_max(code, y, codewords, y_max)))
