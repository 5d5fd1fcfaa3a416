"""Randomized cross-check of the reference decoder against a dense restatement of the method.

For random small codes, samples and parameters (every variant: multi-bit with or without
threshold adaptation and output smoothing, and the single-bit Step 3a), the FP64 reference
decoder must give exactly the decisions, iteration counts and pass flags of a plain numpy
decoder over the dense parity-check matrix (Sec. III-B Steps 1-4, Step 2 of Sec. III-C, Sec.
III-D in the theta lambda^u form of Sec. V-A, Eq. 7 of Sec. III-E), fed the reference decoder's
FP64 perturbations (pinned separately against the library inverse normal CDF).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1402_2773_gb300 import workload as wl

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

CODES = {}


def code_for(n, dv, seed):
    key = (n, dv, seed)
    if key not in CODES:
        CODES[key] = wl.peg_code(n, n // 2, dv, seed=seed)
    return CODES[key]


def dense_decode(O, H, y, w, theta, lam, eta, sigma, T, W, y_max, variant, seed, frame):
    """One frame, FP64, in the order of the paper's steps (flooding schedule)."""
    m, n = H.shape
    adapt, smooth, single = bool(variant & 1), bool(variant & 2), bool(variant & 4)
    v = y.astype(np.float32)
    if y_max > 0:
        v = np.clip(v, np.float32(-y_max), np.float32(y_max))
    ys = v.astype(np.float64)
    x = np.where(v >= 0, 1, -1).astype(np.int64)
    u = np.zeros(n, np.int64)
    Xs = np.zeros(n, np.int64)
    thr = np.array([float(np.float32(theta)) * math.pow(float(np.float32(lam)), k) for k in range(T + 1)])
    scale = float(np.float32(eta)) * float(np.float32(sigma))
    wd = float(np.float32(w))
    t_smooth = max(0, T - W) if smooth else T + 1
    for t in range(T + 1):
        s = np.prod(np.where(H == 1, x[None, :], 1), axis=1)
        if (s == 1).all():
            return x, t, 1
        if t >= t_smooth:
            Xs += x
        if t == T:
            break
        S = H.T.astype(np.int64) @ s
        z = np.concatenate([O.gauss4_f64(seed, frame, t, g) for g in range((n + 3) // 4)])[:n]
        E = (x * ys + wd * S) + scale * z
        if single:
            k = int(np.argmin(E))            # the first index among equal least values
            x[k] = -x[k]
            continue
        flip = E < thr[u]
        if adapt:
            u += ~flip
        x = np.where(flip, -x, x)
    if smooth:
        x = np.where(Xs > 0, 1, np.where(Xs < 0, -1, x))
    return x, T, 0


@settings(max_examples=120, deadline=None, derandomize=True)
@given(n=st.sampled_from([12, 16, 20, 24, 32, 40]), dv=st.sampled_from([2, 3]),
       code_seed=st.integers(1, 3), frames=st.integers(1, 4), data_seed=st.integers(0, 10 ** 6),
       w=st.floats(0.05, 1.5), theta=st.floats(-1.5, 0.0), eta=st.sampled_from([0.0, 0.3, 0.7, 1.0]),
       lam=st.sampled_from([1.0, 0.99, 0.9, 0.8]), T=st.integers(0, 30), W=st.integers(0, 40),
       y_max=st.sampled_from([0.0, 0.8, 2.5]), variant=st.sampled_from([0, 1, 2, 3, 4, 6]),
       sigma=st.floats(0.3, 1.2), seed=st.integers(0, 2 ** 40), frame_offset=st.integers(0, 2 ** 33))
def test_reference_decoder_equals_dense_restatement(n, dv, code_seed, frames, data_seed, w, theta, eta, lam,
                                                     T, W, y_max, variant, sigma, seed, frame_offset):
    O = oracle.load()
    code = code_for(n, dv, code_seed)
    H = code.dense().astype(np.int64)
    rng = np.random.default_rng(data_seed)
    y = (rng.choice([-1.0, 1.0], size=(frames, n)) + sigma * rng.standard_normal((frames, n))).astype(np.float32)
    if variant & 4:
        lam = 1.0                             # Step 3a has no adaptation
    p = oracle.make_params(w=w, theta=theta, eta=eta, lam=lam, y_max=y_max, t_max=T, smooth_window=W,
                           variant=variant)
    bits, iters, ps = O.decode_f64(code, y, sigma, p, seed=seed, frame_offset=frame_offset)
    got = wl.unpack_bits(bits, n)
    for f in range(frames):
        x, t, pa = dense_decode(O, H, y[f], w, theta, lam, eta, sigma, T, W, y_max, variant, seed,
                                frame_offset + f)
        assert iters[f] == t and ps[f] == pa, (f, iters[f], t, ps[f], pa)
        assert (got[f] == (x < 0)).all(), f"frame {f}: decisions differ"
