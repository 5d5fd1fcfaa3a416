"""Randomized cross-check of the reference decoder against a dense restatement of the method.

For random small codes, samples and parameters (every variant: multi-bit with or without
threshold adaptation and output smoothing, and the single-bit Step 3a, with Gaussian or uniform
perturbations) and every arithmetic (FP64, FP32, binary16, Q-bit fixed point of Eq. 8, and Q-bit
held samples with the fine fixed-point accumulator), the reference decoder must give exactly the
decisions, iteration counts and pass flags of a plain numpy decoder over the dense parity-check
matrix (Sec. III-B Steps 1-4, Step 2 of Sec. III-C, Sec. III-D in the theta lambda^u form of
Sec. V-A, Eq. 7 of Sec. III-E).  The numpy decoder takes from the reference decoder only what is
pinned separately: the perturbation deviates (library inverse normal CDF), the FP32 threshold
table (closed form) and the fixed-point scale.
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


def f16(a):
    """Rounded to binary16 (nearest even) and back to FP32."""
    return np.asarray(a, np.float32).astype(np.float16).astype(np.float32)


def fix_value(a, R, kmax):
    """Eq. 8 level value 2b + 1 (units of Delta/2), the level decided in FP32."""
    a = np.asarray(a, np.float32)
    k = np.floor(np.abs(a) * np.float32(R))
    k = np.where(k < kmax, k, kmax).astype(np.int64)
    return np.where(a >= 0, 2 * k + 1, -2 * k - 1)


def dense_decode(O, H, y, w, theta, lam, eta, sigma, T, W, y_max, variant, seed, frame, prec, q_bits):
    """One frame in the order of the paper's steps (flooding schedule)."""
    m, n = H.shape
    adapt, smooth, single = bool(variant & 1), bool(variant & 2), bool(variant & 4)
    uniform = bool(variant & 8)
    v = y.astype(np.float32)
    if y_max > 0:
        v = np.clip(v, np.float32(-y_max), np.float32(y_max))
    if prec == "f16":
        v = f16(v)
    ys = v.astype(np.float64)
    x = np.where(v >= 0, 1, -1).astype(np.int64)
    u = np.zeros(n, np.int64)
    Xs = np.zeros(n, np.int64)
    if prec == "f64":
        thr = np.array([float(np.float32(theta)) * math.pow(float(np.float32(lam)), k) for k in range(T + 1)])
        scale = float(np.float32(eta)) * float(np.float32(sigma))
        if uniform:
            scale *= math.sqrt(3.0)
        wd = float(np.float32(w))
    else:
        thr = O.threshold_table_f32(theta, lam, T)
        scale = float(np.float32(eta)) * float(np.float32(sigma))
        scale = np.float32(scale * math.sqrt(3.0) if uniform else scale)
        wd = np.float32(w)
        if prec == "f16":
            thr, wd = f16(thr), f16(wd)
        if prec == "fix":
            R, kmax = O.fix_scale(q_bits, y_max), 2 ** (q_bits - 1) - 1
            yq = fix_value(v, R, kmax)
            x = np.where(yq > 0, 1, -1).astype(np.int64)
            thr = fix_value(thr, R, kmax)
            wq = int(fix_value(wd, R, kmax))
        if prec == "acc":
            R, kmax = O.fix_scale(q_bits, y_max), 2 ** (q_bits - 1) - 1
            Rd = np.float32(O.fixacc_scale(q_bits, y_max))
            yq = fix_value(v, R, kmax)
            x = np.where(yq > 0, 1, -1).astype(np.int64)
            thr = np.rint(np.asarray(thr, np.float32) * Rd).astype(np.int64)
            wq = int(np.rint(np.float32(wd) * Rd))
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
        if uniform:
            zu = np.concatenate([O.uniform4_f32(seed, frame, t, g) for g in range((n + 3) // 4)])[:n]
        if prec == "f64":
            z = zu.astype(np.float64) if uniform else \
                np.concatenate([O.gauss4_f64(seed, frame, t, g) for g in range((n + 3) // 4)])[:n]
            E = (x * ys + wd * S) + scale * z
        else:
            z = zu if uniform else np.concatenate([O.gauss4_f32(seed, frame, t, g) for g in range((n + 3) // 4)])[:n]
            q = (scale * z).astype(np.float32)
            xy = np.where(x > 0, v, -v).astype(np.float32)
            if prec == "f32":
                E = (xy + wd * S.astype(np.float32)) + q
            elif prec == "f16":
                E = f16(f16(xy + f16(wd * S.astype(np.float32))) + f16(q))
            elif prec == "acc":
                E = x * yq * 256 + wq * S + np.rint(q * Rd).astype(np.int64)
            else:
                E = x * yq + wq * S + fix_value(q, R, kmax)
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


@settings(max_examples=200, deadline=None, derandomize=True)
@given(n=st.sampled_from([12, 16, 20, 24, 32, 40]), dv=st.sampled_from([2, 3]),
       code_seed=st.integers(1, 3), frames=st.integers(1, 4), data_seed=st.integers(0, 10 ** 6),
       w=st.floats(0.05, 1.5), theta=st.floats(-1.5, 0.0), eta=st.sampled_from([0.0, 0.3, 0.7, 1.0]),
       lam=st.sampled_from([1.0, 0.99, 0.9, 0.8]), T=st.integers(0, 30), W=st.integers(0, 40),
       y_max=st.sampled_from([0.0, 0.8, 2.5]), variant=st.sampled_from([0, 1, 2, 3, 4, 6, 8, 11, 12]),
       sigma=st.floats(0.3, 1.2), seed=st.integers(0, 2 ** 40), frame_offset=st.integers(0, 2 ** 33),
       prec=st.sampled_from(["f64", "f32", "f16", "fix", "acc"]), q_bits=st.integers(2, 8))
def test_reference_decoder_equals_dense_restatement(n, dv, code_seed, frames, data_seed, w, theta, eta, lam,
                                                     T, W, y_max, variant, sigma, seed, frame_offset, prec,
                                                     q_bits):
    O = oracle.load()
    if prec in ("fix", "acc") and y_max == 0.0:
        y_max = 2.0                           # the fixed point needs a saturation level
    code = code_for(n, dv, code_seed)
    H = code.dense().astype(np.int64)
    rng = np.random.default_rng(data_seed)
    y = (rng.choice([-1.0, 1.0], size=(frames, n)) + sigma * rng.standard_normal((frames, n))).astype(np.float32)
    if variant & 4:
        lam = 1.0                             # Step 3a has no adaptation
    precision = {"f64": oracle.FP32, "f32": oracle.FP32, "f16": oracle.FP16, "fix": oracle.FIX,
                 "acc": oracle.FIXACC}[prec]
    p = oracle.make_params(w=w, theta=theta, eta=eta, lam=lam, y_max=y_max, t_max=T, smooth_window=W,
                           variant=variant, precision=precision, q_bits=q_bits if prec in ("fix", "acc") else 0)
    decode = O.decode_f64 if prec == "f64" else O.decode_f32
    bits, iters, ps = decode(code, y, sigma, p, seed=seed, frame_offset=frame_offset)
    got = wl.unpack_bits(bits, n)
    for f in range(frames):
        x, t, pa = dense_decode(O, H, y[f], w, theta, lam, eta, sigma, T, W, y_max, variant, seed,
                                frame_offset + f, prec, q_bits)
        assert iters[f] == t and ps[f] == pa, (f, iters[f], t, ps[f], pa)
        assert (got[f] == (x < 0)).all(), f"frame {f}: decisions differ"


@settings(max_examples=400, deadline=None, derandomize=True)
@given(x=st.sampled_from([1, -1]), ys=st.floats(-3.0, 3.0, width=32), S=st.integers(-12, 12),
       w=st.floats(0.0, 2.0, width=32), q=st.floats(-4.0, 4.0, width=32))
def test_inversion_function_forms_equal_their_definitions(x, ys, S, w, q):
    """E_k = ((x_k y_k) + w S_k) + q_k in each arithmetic, bit for bit: FP32 and FP64 with one
    rounding per operation in this order, binary16 with every result rounded to binary16."""
    O = oracle.load()
    f32 = np.float32
    xy = f32(ys) if x > 0 else -f32(ys)
    want32 = (xy + f32(w) * f32(S)) + f32(q)
    assert np.float32(O.metric_f32(x, ys, S, w, q)).tobytes() == want32.tobytes()
    ys16, w16 = float(f16(ys)), float(f16(w))
    xy16 = f16(ys16 if x > 0 else -ys16)
    want16 = f16(f16(xy16 + f16(f32(w16) * f32(S))) + f16(q))
    assert np.float32(O.metric_f16(x, ys16, S, w16, q)).tobytes() == np.float32(want16).tobytes()
    want64 = ((float(ys) if x > 0 else -float(ys)) + float(w) * S) + float(q)
    assert O.metric_f64(x, float(ys), S, float(w), float(q)) == want64
