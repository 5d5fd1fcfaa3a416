"""Pins of the reference (oracle) decoder to facts outside the oracle itself.

Each ``pin_*`` function takes an ``oracle.Oracle`` and raises AssertionError
when the oracle disagrees with the paper (Sundararajan, Winstead, Boutillon
2014), with a closed form, with a library routine evaluating a textbook
definition, with an invariant, or with a trace worked out by hand.  The
test modules run every pin on the real oracle, and run the whole battery
on oracles with planted mistakes, each of which must fail at least one pin.
"""
from __future__ import annotations

import math
import os

import numpy as np

import oracle as oracle_pkg
from paper_1402_2773_gb300 import workload as wl

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden_lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


# ---------------------------------------------------------------------------
# tiny codes
# ---------------------------------------------------------------------------

# Hamming (7,4): N(0) = {0,1,3,4}, N(1) = {0,2,3,5}, N(2) = {1,2,3,6};
# M(0) = {0,1}, M(1) = {0,2}, M(2) = {1,2}, M(3) = {0,1,2}, M(4..6) = {0},{1},{2}.
HAMMING_H = np.array([[1, 1, 0, 1, 1, 0, 0],
                      [1, 0, 1, 1, 0, 1, 0],
                      [0, 1, 1, 1, 0, 0, 1]], dtype=np.uint8)


def hamming_code():
    return wl.code_from_dense(HAMMING_H, name="hamming74")


def _bits_byte(bits):
    return int(bits[0])


# ---------------------------------------------------------------------------
# generator
# ---------------------------------------------------------------------------

def pin_philox_kat(O):
    """Philox4x32-10 against the authors' published known-answer vectors."""
    for row in _golden_lines("philox4x32_10_kat.txt"):
        v = [int(h, 16) for h in row]
        got = O.philox(v[0:4], v[4:6])
        assert list(got) == v[6:10], f"philox KAT mismatch: {got} vs {v[6:10]}"


def _icdf_inputs():
    """Philox outputs covering every segment densely: for each level j (leading zeros of
    a = 2 (r mod 2^31) + 1) and sub-interval s, 1024 evenly spaced positions plus both ends,
    and 2^18 uniformly random outputs; both signs."""
    rng = np.random.default_rng(11)
    rs = [rng.integers(0, 1 << 32, 1 << 18, dtype=np.uint64)]
    for j in range(32):
        lo, hi = (1 << (31 - j)), (1 << (32 - j))          # a in [lo, hi): j leading zeros
        a = np.unique(np.concatenate([np.linspace(lo, hi - 1, 8 * 1024 + 1).astype(np.uint64),
                                      lo + (hi - lo) // 8 * np.arange(8, dtype=np.uint64),
                                      lo + (hi - lo) // 8 * np.arange(1, 9, dtype=np.uint64) - 1]))
        a = a | np.uint64(1)
        r = (a - np.uint64(1)) // np.uint64(2)
        rs += [r, r | np.uint64(1 << 31)]
    return np.unique(np.concatenate(rs)).astype(np.uint32)


def _ndtri_of(r):
    from scipy.special import ndtri
    r = r.astype(np.uint64)
    p = (2.0 * (r & np.uint64(0x7FFFFFFF)).astype(np.float64) + 1.0) * 2.0 ** -33
    z = ndtri(p)
    return np.where(r >> np.uint64(31) == 1, -z, z)


def pin_icdf_vs_library(O):
    """FP32 inverse-CDF deviate of every segment within 2.5 ulp of max(|z|, 1) of the library's
    Phi^{-1} (scipy ndtri) at p = (2 (r mod 2^31) + 1) 2^-33, sign from bit 31."""
    r = _icdf_inputs()
    z = O.gauss_many_f32(r).astype(np.float64)
    assert all(z[i] == O.gauss_f32(int(r[i])) for i in range(0, len(r), len(r) // 50))
    ref = _ndtri_of(r)
    ulp = np.spacing(np.maximum(np.abs(ref), 1.0).astype(np.float32)).astype(np.float64)
    worst = float(np.max(np.abs(z - ref) / ulp))
    assert worst <= 2.5, f"FP32 deviate off the library inverse CDF by {worst} ulp"
    # the batch evaluator over consecutive outputs agrees, around segment and level edges
    for start in (0, (1 << 30) - 64, (1 << 31) - 64, 0x80000000 - 64, 0xFFFFFFFF - 127, 12345678):
        zz = O.gauss_range_f32(start, 128).astype(np.float64)
        rr = (start + np.arange(128, dtype=np.uint64)).astype(np.uint32)
        ref = _ndtri_of(rr)
        ulp = np.spacing(np.maximum(np.abs(ref), 1.0).astype(np.float32)).astype(np.float64)
        assert np.max(np.abs(zz - ref) / ulp) <= 2.5


def pin_icdf_symmetry_and_range(O):
    """z(r with bit 31 set) = -z(r) exactly; the extreme outputs give Phi^{-1}(2^-33) = -6.3379."""
    for r in (0, 1, 77, 1 << 20, (1 << 30) + 5, (1 << 31) - 1):
        assert O.gauss_f32(r | (1 << 31)) == -O.gauss_f32(r)
        assert O.gauss_f64(r | (1 << 31)) == -O.gauss_f64(r)
    assert abs(float(O.gauss_f32(0)) + 6.33795775455) < 1e-6
    assert abs(O.gauss_f64(0) + 6.337957754553) < 1e-11


def pin_gauss_f64_vs_library(O):
    """The FP64 deviate equals the library's Phi^{-1} to 1e-13 (absolute, |z| <= 6.4)."""
    r = _icdf_inputs()[::97]
    z = np.array([O.gauss_f64(int(v)) for v in r])
    assert np.max(np.abs(z - _ndtri_of(r))) < 1e-13


def pin_gauss4_wiring(O):
    """Symbol 4g + i takes Philox output i of counter (g, t, frame_lo, frame_hi), key (seed_lo, seed_hi)."""
    for seed, f, t, g in ((12345, 0, 0, 0), (7, 3, 299, 511), ((5 << 32) | 9, (2 << 32) | 1, 17, 3)):
        r = O.philox([g, t, f & 0xFFFFFFFF, f >> 32], [seed & 0xFFFFFFFF, seed >> 32])
        z32 = O.gauss4_f32(seed, f, t, g)
        z64 = O.gauss4_f64(seed, f, t, g)
        for i in range(4):
            assert z32[i] == O.gauss_f32(int(r[i])) and z64[i] == O.gauss_f64(int(r[i]))


def pin_gauss_statistics(O):
    """z ~ N(0,1): Kolmogorov-Smirnov, first moments, pair independence, radial law."""
    from scipy import stats
    z = np.array([O.gauss4_f64(7, f, t, g) for f in range(16) for t in range(8) for g in range(64)])
    zz = z.reshape(-1)
    assert stats.kstest(zz, "norm").pvalue > 1e-4, "Gaussian KS test"
    assert abs(zz.mean()) < 0.02 and abs(zz.var() - 1.0) < 0.03
    assert abs(np.corrcoef(z[:, 0], z[:, 1])[0, 1]) < 0.03
    r2 = z[:, 0] ** 2 + z[:, 1] ** 2          # chi-square with 2 dof: exponential, mean 2
    assert stats.kstest(r2, "expon", args=(0, 2)).pvalue > 1e-4
    z32 = np.array([O.gauss4_f32(7, f, t, g) for f in range(16) for t in range(8) for g in range(64)],
                   dtype=np.float64).reshape(-1)
    assert stats.kstest(z32, "norm").pvalue > 1e-4


def pin_noise_variance(O):
    """q_k has standard deviation eta * sigma (Sec. III-C; N0/2 = sigma^2)."""
    eta, sigma = 0.7, 0.6
    q = np.array([O.noise_f32(3, f, t, k, eta, sigma) for f in range(4) for t in range(16)
                  for k in range(256)], dtype=np.float64)
    sd = q.std()
    assert abs(sd - eta * sigma) < 0.02 * eta * sigma, f"perturbation std {sd}"
    assert abs(q.mean()) < 0.02


# ---------------------------------------------------------------------------
# thresholds, quantizer, inversion function
# ---------------------------------------------------------------------------

def pin_threshold_table(O):
    """theta_k = theta lambda^u (Sec. V-A, Eq. 12): within 1 FP32 ulp of the closed form."""
    for theta, lam, T in ((-0.9, 0.99, 300), (-0.7, 0.993, 300), (-0.6, 1.0, 50), (-0.9, 0.9, 100)):
        thr = O.threshold_table_f32(theta, lam, T)
        ref = float(np.float32(theta)) * float(np.float32(lam)) ** np.arange(T + 1, dtype=np.float64)
        err = np.abs(thr.astype(np.float64) - ref) / np.spacing(np.abs(ref).astype(np.float32))
        assert err.max() <= 1.0, f"threshold table off by {err.max()} ulp"


def pin_table2(O):
    """Quantized adaptation events reproduce Table II of Sec. V-A exactly."""
    want = {}
    for q, i, th, tau in _golden_lines("table2_threshold_events.txt"):
        want.setdefault(int(q), []).append((float(th), int(tau)))
    for q, events in want.items():
        got = O.threshold_events(-0.9, 0.99, 300, q, 2.5)
        assert len(got) == len(events), f"Q={q}: {got}"
        for (gth, gtau), (wth, wtau) in zip(got, events):
            assert gtau == wtau and round(gth, 4) == wth, f"Q={q}: {got} vs {events}"


def pin_fig20(O):
    """Weighted-GDBF flip matrices of Fig. 20 (Sec. VII) from the oracle's inversion function."""
    lines = _golden_lines("fig20_weighted_flip_matrices.txt")
    mats, cur = {}, None
    for ln in lines:
        if ln[0] == "theta":
            cur = float(ln[1])
            mats[cur] = []
        else:
            mats[cur].append([int(v) for v in ln])
    nq = 16
    rows = [O.quantize((k + 0.5) * 3.0 / nq, 4, 1.5) for k in range(nq // 2 - 1, -1, -1)]
    assert rows[0] == 1.40625 and rows[-1] == 0.09375
    for theta, want in mats.items():
        for r, ys in enumerate(rows):
            for c, S in enumerate((3, 1, -1, -3)):
                e = O.metric_f32(+1, ys, S, 0.5, 0.0)
                got = -1 if e < np.float32(theta) else 1
                assert got == want[r][c], f"theta={theta} row {r} col {c}"
                e64 = O.metric_f64(+1, ys, S, 0.5, 0.0)
                assert (-1 if e64 < theta else 1) == want[r][c]


def pin_quantizer(O):
    """g(.) of Eq. 8: odd multiples of Delta/2, saturating at +-(N_Q - 1) Delta / 2."""
    for q in (3, 4, 5, 8):
        d = 2 * 2.5 / 2 ** q
        for v in np.linspace(-4, 4, 801):
            g = O.quantize(float(v), q, 2.5)
            k = (abs(g) / d) - 0.5
            assert abs(k - round(k)) < 1e-9 and 0 <= round(k) <= 2 ** (q - 1) - 1
            if abs(v) < 2.5 - 1e-9:
                assert abs(g - v) <= d / 2 + 1e-12
            assert (g > 0) == (v >= 0)


# ---------------------------------------------------------------------------
# decoder: hand-worked traces on the Hamming (7,4) code
# ---------------------------------------------------------------------------

Y_A = np.array([0.8, 0.9, 1.1, -0.2, 0.7, 1.0, 0.6], dtype=np.float32)


def pin_trace_gdbf(O):
    """Case A: s = (-1,-1,-1) at t = 0; with w = 0.5, theta = -0.6:
    E = (-0.2, -0.1, 0.1, -1.3, 0.2, 0.5, 0.1) so only x_3 flips; t = 1 is valid."""
    C = hamming_code()
    p = oracle_pkg.make_params(w=0.5, theta=-0.6, eta=0.0, lam=1.0, y_max=2.5, t_max=10)
    bits, it, ps = O.decode_f32_qin(C, Y_A, p, np.zeros((10, 7), np.float32))
    assert (_bits_byte(bits), it, ps) == (0, 1, 1)
    # T = 1 still allows the single flip phase; T = 0 tests x(0) only
    p1 = oracle_pkg.make_params(w=0.5, theta=-0.6, eta=0.0, lam=1.0, y_max=2.5, t_max=1)
    assert (lambda r: (_bits_byte(r[0]), r[1], r[2]))(O.decode_f32_qin(C, Y_A, p1, np.zeros((1, 7), np.float32))) == (0, 1, 1)
    p0 = oracle_pkg.make_params(w=0.5, theta=-0.6, eta=0.0, lam=1.0, y_max=2.5, t_max=0)
    bits, it, ps = O.decode_f32_qin(C, Y_A, p0, np.zeros((0, 7), np.float32))
    assert (_bits_byte(bits), it, ps) == (0x08, 0, 0)


def pin_trace_injected_noise(O):
    """Case B: q_4(0) = -1 pushes E_4 = 0.2 - 1.0 = -0.8 below theta: x_3 and x_4 flip at t = 0.
    At t = 1, s = (-1, +1, +1), E_4 = -0.7 - 0.5 = -1.2 flips x_4 back; t = 2 is valid."""
    C = hamming_code()
    p = oracle_pkg.make_params(w=0.5, theta=-0.6, eta=0.0, lam=1.0, y_max=2.5, t_max=10)
    q = np.zeros((10, 7), np.float32)
    q[0, 4] = -1.0
    bits, it, ps = O.decode_f32_qin(C, Y_A, p, q)
    assert (_bits_byte(bits), it, ps) == (0, 2, 1)
    # With q_4(0) = -0.1 instead, E_4 = 0.1 > theta: the trace of case A.
    q[0, 4] = -0.1
    bits, it, ps = O.decode_f32_qin(C, Y_A, p, q)
    assert (_bits_byte(bits), it, ps) == (0, 1, 1)


def pin_trace_adaptation(O):
    """Case C: y_3 = -0.1, w = 0.2, theta = -0.6.  t = 0: E_3 = 0.1 - 0.6 = -0.5 >= -0.6, no flip,
    every u_k = 1.  With lambda = 0.5 the threshold becomes -0.3 and E_3 = -0.5 flips at t = 1,
    so t = 2 is valid.  Without adaptation x never changes: T is reached with x_3 = -1."""
    C = hamming_code()
    y = Y_A.copy()
    y[3] = -0.1
    pa = oracle_pkg.make_params(w=0.2, theta=-0.6, eta=0.0, lam=0.5, y_max=2.5, t_max=6,
                                variant=oracle_pkg.ADAPT)
    bits, it, ps = O.decode_f32_qin(C, y, pa, np.zeros((6, 7), np.float32))
    assert (_bits_byte(bits), it, ps) == (0, 2, 1)
    pn = oracle_pkg.make_params(w=0.2, theta=-0.6, eta=0.0, lam=0.5, y_max=2.5, t_max=6, variant=0)
    bits, it, ps = O.decode_f32_qin(C, y, pn, np.zeros((6, 7), np.float32))
    assert (_bits_byte(bits), it, ps) == (0x08, 6, 0)


def pin_trace_smoothing(O):
    """Case D: T = 4, W = 3 (window t = 1..4), q = -5 forces a flip and +5 forbids one.
    Flips: t=1 {3,4}, t=2 {5}, t=3 {0,3}.  x(1) = (+,+,+,-,+,+,+), x(2) = (+,+,+,+,-,+,+),
    x(3) = (+,+,+,+,-,-,+), x(4) = (-,+,+,-,-,-,+); no x(t) satisfies all checks.
    Window sums X = (2,4,4,0,-2,0,4): smoothed output (+,+,+,-,-,-,+) (zeros keep x(4)),
    bits 3,4,5 -> 0x38; unsmoothed output x(4) -> 0x39."""
    C = hamming_code()
    q = np.full((4, 7), 5.0, np.float32)
    for t, k in ((1, 3), (1, 4), (2, 5), (3, 3), (3, 0)):
        q[t, k] = -5.0
    ps_ = oracle_pkg.make_params(w=0.5, theta=-0.6, eta=0.0, lam=1.0, y_max=2.5, t_max=4,
                                 smooth_window=3, variant=oracle_pkg.SMOOTH)
    bits, it, ps = O.decode_f32_qin(C, Y_A, ps_, q)
    assert (_bits_byte(bits), it, ps) == (0x38, 4, 0)
    pn = oracle_pkg.make_params(w=0.5, theta=-0.6, eta=0.0, lam=1.0, y_max=2.5, t_max=4,
                                smooth_window=3, variant=0)
    bits, it, ps = O.decode_f32_qin(C, Y_A, pn, q)
    assert (_bits_byte(bits), it, ps) == (0x39, 4, 0)


def pin_trace_clamp_sign_tie(O):
    """Case F: saturation at Y_max = 2 turns E_3 = 2.8 - 3 = -0.2 into 2 - 3 = -1 < -0.6 (w = 1).
    Case G: y_3 = 0 gives x_3 = +1 and the all-(+1) word is valid at t = 0.
    Case H: y_3 = -0.25, w = 0.25, theta = -0.5: E_3 = 0.25 - 0.75 = -0.5 = theta exactly, no flip."""
    C = hamming_code()
    y = np.array([2.0, 2.0, 2.0, -2.8, 0.7, 1.0, 0.6], np.float32)
    p = oracle_pkg.make_params(w=1.0, theta=-0.6, eta=0.0, lam=1.0, y_max=2.0, t_max=5)
    bits, it, ps = O.decode_f32_qin(C, y, p, np.zeros((5, 7), np.float32))
    assert (_bits_byte(bits), it, ps) == (0, 1, 1)
    p_noclamp = oracle_pkg.make_params(w=1.0, theta=-0.6, eta=0.0, lam=1.0, y_max=math.inf, t_max=5)
    bits, it, ps = O.decode_f32_qin(C, y, p_noclamp, np.zeros((5, 7), np.float32))
    assert (_bits_byte(bits), it, ps) == (0x08, 5, 0)
    y0 = Y_A.copy()
    y0[3] = 0.0
    p = oracle_pkg.make_params(w=0.5, theta=-0.6, eta=0.0, lam=1.0, y_max=2.5, t_max=5)
    bits, it, ps = O.decode_f32_qin(C, y0, p, np.zeros((5, 7), np.float32))
    assert (_bits_byte(bits), it, ps) == (0, 0, 1)
    yt = Y_A.copy()
    yt[3] = -0.25
    p = oracle_pkg.make_params(w=0.25, theta=-0.5, eta=0.0, lam=1.0, y_max=2.5, t_max=3)
    bits, it, ps = O.decode_f32_qin(C, yt, p, np.zeros((3, 7), np.float32))
    assert (_bits_byte(bits), it, ps) == (0x08, 3, 0)


# ---------------------------------------------------------------------------
# decoder: invariants and special cases on seeded codes
# ---------------------------------------------------------------------------

def _pin_code():
    return wl.peg_code(96, 48, 3, seed=11)


def pin_trace_single_bit(O):
    """Case J (Step 3a), dyadic samples y = (0.75, 0.875, 1.125, -0.25, 0.75, 1, 0.625), w = 0.5.
    t = 0, s = (-1,-1,-1): E = (-0.25, -0.125, 0.125, -1.25, 0.25, 0.5, 0.125); argmin k = 3 alone,
    so x_3 flips and t = 1 is valid (output 0, 1 iteration).  With q_0(0) = -1 the least value
    -1.25 is shared by k = 0 and k = 3 and goes to the lower index: x_0 flips, x(1) = (-,+,+,-,+,+,+)
    gives s = (+1,+1,-1) and E = (0.25, 0.875, 1.125, 0.75, 1.25, 1.5, 0.125), so x_6 flips and
    t = 2 is valid with the codeword whose bits 0, 3, 6 are set (0x49)."""
    C = hamming_code()
    y = np.array([0.75, 0.875, 1.125, -0.25, 0.75, 1.0, 0.625], np.float32)
    p = oracle_pkg.make_params(w=0.5, theta=-0.6, eta=0.0, lam=1.0, y_max=2.5, t_max=10, variant=oracle_pkg.SINGLE)
    bits, it, ps = O.decode_f32_qin(C, y, p, np.zeros((10, 7), np.float32))
    assert (_bits_byte(bits), it, ps) == (0, 1, 1)
    q = np.zeros((10, 7), np.float32)
    q[0, 0] = -1.0
    bits, it, ps = O.decode_f32_qin(C, y, p, q)
    assert (_bits_byte(bits), it, ps) == (0x49, 2, 1)


def _sgdbf_dense(H, y, w, T, y_max):
    """Textbook S-GDBF (Wadayama et al. 2010, single-bit): flip argmin E_k (first on ties), FP64."""
    ys = np.clip(y.astype(np.float64), -y_max, y_max)
    x = np.where(ys >= 0, 1, -1)
    Hi = H.astype(np.int64)
    for t in range(T + 1):
        s = 1 - 2 * ((Hi @ (x < 0).astype(np.int64)) % 2)
        if (s == 1).all():
            return x, t, 1
        if t == T:
            break
        E = x * ys + w * (Hi.T @ s)
        k = int(np.argmin(E))
        x[k] = -x[k]
    return x, T, 0


def pin_eta0_is_single_bit_gdbf(O):
    """eta = 0 with the single-bit variant equals textbook S-GDBF evaluated densely."""
    C = _pin_code()
    H = C.dense()
    y, _, sig = wl.frames(C, 60, 3.0, seed=19)
    p = oracle_pkg.make_params(w=0.75, theta=-0.9, eta=0.0, lam=1.0, y_max=2.5, t_max=60, variant=oracle_pkg.SINGLE)
    bits, it, ps = O.decode_f64(C, y, sig, p, seed=1)
    xs = wl.unpack_bits(bits, C.n)
    for f in range(y.shape[0]):
        x, t, pa = _sgdbf_dense(H, y[f], float(np.float32(0.75)), 60, 2.5)
        assert it[f] == t and ps[f] == pa and (xs[f] == (x < 0)).all(), f"frame {f}"
    assert (ps == 1).any() and (ps == 0).any()


def pin_noiseless(O):
    """A transmitted codeword (y = 1 - 2c) satisfies every check: iters = 0, pass = 1, output c."""
    C = _pin_code()
    y, cw, _ = wl.frames(C, 16, None, seed=3)
    for variant in (0, 1, 3):
        p = oracle_pkg.make_params(variant=variant, t_max=20, smooth_window=8)
        for dec in (O.decode_f32, O.decode_f64):
            bits, it, ps = dec(C, y, 0.5, p, seed=1)
            assert (it == 0).all() and (ps == 1).all() and (bits == cw).all()


def _mgdbf_dense(H, y, w, theta, lam, T, y_max, adapt):
    """Textbook M-GDBF / AT-GDBF (Wadayama et al. 2010; Ismail et al. 2013) on a dense H, FP64."""
    ys = np.clip(y.astype(np.float64), -y_max, y_max)
    x = np.where(ys >= 0, 1, -1)
    thr = np.full(H.shape[1], theta, dtype=np.float64)
    Hi = H.astype(np.int64)
    for t in range(T + 1):
        s = 1 - 2 * ((Hi @ (x < 0).astype(np.int64)) % 2)
        if (s == 1).all():
            return x, t, 1
        if t == T:
            break
        E = x * ys + w * (Hi.T @ s)
        flip = E < thr
        x = np.where(flip, -x, x)
        if adapt:
            thr = np.where(flip, thr, thr * lam)
    return x, T, 0


def pin_eta0_is_gdbf(O):
    """eta = 0 removes the perturbation: the oracle equals textbook M-GDBF (lambda = 1) and
    AT-GDBF (lambda < 1) evaluated densely."""
    C = _pin_code()
    H = C.dense()
    y, _, sig = wl.frames(C, 60, 2.5, seed=9)
    for lam, adapt, w, theta in ((1.0, 0, 0.75, -0.9), (0.9, 1, 0.5, -0.7), (0.97, 1, 1.0, -1.2)):
        p = oracle_pkg.make_params(w=w, theta=theta, eta=0.0, lam=lam, y_max=2.5, t_max=40,
                                   variant=oracle_pkg.ADAPT if adapt else 0)
        bits, it, ps = O.decode_f64(C, y, sig, p, seed=1)
        b32, it32, ps32 = O.decode_f32(C, y, sig, p, seed=1)
        xs = wl.unpack_bits(bits, C.n)
        same = 0
        for f in range(y.shape[0]):
            x, t, pa = _mgdbf_dense(H, y[f], float(np.float32(w)), float(np.float32(theta)),
                                    float(np.float32(lam)), 40, 2.5, adapt)
            ok = (it[f] == t and ps[f] == pa and (xs[f] == (x < 0)).all())
            same += ok
        assert same == y.shape[0], f"eta=0 oracle differs from textbook GDBF on {y.shape[0] - same} frames"
        assert (it32 == it).mean() > 0.95


def pin_codeword_and_ml(O):
    """N = 24 brute force: a passing output is a codeword (dense H x = 0); NGDBF cannot beat ML."""
    C = wl.peg_code(24, 12, 3, seed=2)
    H = C.dense().astype(np.int64)
    enc = C.encoder()
    K = enc.k
    infos = ((np.arange(2 ** K)[:, None] >> np.arange(K)[None, :]) & 1).astype(np.uint8)
    cws = np.zeros((2 ** K, C.n), np.uint8)
    cws[:, enc.info_pos] = infos
    pm = wl.unpack_bits(enc.pmask.view(np.uint8).reshape(enc.rank, -1), enc.pmask.shape[1] * 64)[:, :K]
    cws[:, enc.pivot_pos] = (infos.astype(np.int64) @ pm.T.astype(np.int64)) % 2
    assert ((cws.astype(np.int64) @ H.T) % 2 == 0).all()
    y, cw, sig = wl.frames(C, 400, 3.0, seed=4)
    p = oracle_pkg.make_params(w=0.75, theta=-0.9, eta=0.96, lam=0.95, t_max=60, variant=oracle_pkg.ADAPT)
    bits, it, ps = O.decode_f32(C, y, sig, p, seed=8)
    out = wl.unpack_bits(bits, C.n).astype(np.int64)
    synd = (out @ H.T) % 2
    assert (synd[ps == 1] == 0).all(), "a passing frame is not a codeword"
    assert synd[ps == 0].any(axis=1).all(), "a failing (unsmoothed) frame satisfies every check"
    bip = 1.0 - 2.0 * cws.astype(np.float64)
    ml = np.argmax(y.astype(np.float64) @ bip.T, axis=1)
    tx = wl.unpack_bits(cw, C.n)
    ml_err = (cws[ml] != tx).any(axis=1).mean()
    dec_err = (out != tx).any(axis=1).mean()
    n = y.shape[0]
    assert dec_err >= ml_err - 3 * math.sqrt(max(ml_err, 1.0 / n) / n), (dec_err, ml_err)
    corr = (1.0 - 2.0 * out) @ y.T.astype(np.float64)
    corr_ml = np.max(y.astype(np.float64) @ bip.T, axis=1)
    assert (np.diag(corr)[ps == 1] <= corr_ml[ps == 1] + 1e-9).all()


def pin_f32_matches_injected_noise(O):
    """The FP32 decoder adds exactly q_k = noise(seed, frame, t, k) each iteration."""
    C = hamming_code()
    y = np.array([0.3, -0.2, 0.5, 0.1, -0.4, 0.9, -0.05], np.float32)
    for variant, lam in ((0, 1.0), (3, 0.9)):
        p = oracle_pkg.make_params(w=0.5, theta=-0.3, eta=0.9, lam=lam, t_max=12, smooth_window=5,
                                   variant=variant)
        sigma = 0.7
        for fid in range(6):
            q = np.array([[O.noise_f32(99, fid, t, k, 0.9, sigma) for k in range(7)] for t in range(12)],
                         np.float32)
            b1, it1, ps1 = O.decode_f32_qin(C, y, p, q)
            b2, it2, ps2 = O.decode_f32(C, y[None, :], sigma, p, seed=99, frame_offset=fid)
            assert (b1 == b2[0]).all() and it1 == it2[0] and ps1 == ps2[0]
    # frames of a batch are keyed by frame_offset + index, at low SNR where the noise decides
    C = _pin_code()
    y, _, sig = wl.frames(C, 6, 1.0, seed=12)
    p = oracle_pkg.make_params(w=0.75, theta=-0.9, eta=0.96, lam=0.97, t_max=25, variant=1)
    b2, it2, ps2 = O.decode_f32(C, y, sig, p, seed=5, frame_offset=40)
    for f in range(6):
        q = np.array([[O.noise_f32(5, 40 + f, t, k, 0.96, sig) for k in range(C.n)] for t in range(25)],
                     np.float32)
        b1, it1, ps1 = O.decode_f32_qin(C, y[f], p, q)
        assert (b1 == b2[f]).all() and it1 == it2[f] and ps1 == ps2[f], f"frame {f}"


def pin_frame_independence(O):
    """A frame's result depends only on (y, seed, frame id): not on batch position or threads."""
    C = _pin_code()
    y, _, sig = wl.frames(C, 40, 2.0, seed=5)
    p = oracle_pkg.make_params(variant=3, t_max=30, smooth_window=10, lam=0.95)
    b, it, ps = O.decode_f32(C, y, sig, p, seed=4, frame_offset=100, threads=1)
    b2, it2, ps2 = O.decode_f32(C, y[10:20], sig, p, seed=4, frame_offset=110, threads=3)
    assert (b[10:20] == b2).all() and (it[10:20] == it2).all() and (ps[10:20] == ps2).all()
    b3, it3, ps3 = O.decode_f32(C, y, sig, p, seed=4, frame_offset=100, threads=7)
    assert (b == b3).all() and (it == it3).all()


def pin_f32_f64_statistics(O):
    """FP32 and FP64 forms decode the same frames to statistically equal results."""
    C = _pin_code()
    y, cw, sig = wl.frames(C, 300, 3.0, seed=6)
    p = oracle_pkg.make_params(w=0.75, theta=-0.9, eta=0.9, lam=0.95, t_max=50, variant=1)
    b32, it32, ps32 = O.decode_f32(C, y, sig, p, seed=2)
    b64, it64, ps64 = O.decode_f64(C, y, sig, p, seed=2)
    assert (it32 == it64).mean() > 0.8
    assert abs(ps32.mean() - ps64.mean()) < 0.05


# ---------------------------------------------------------------------------
# reduced-precision forms (Sec. IV-E)
# ---------------------------------------------------------------------------

def pin_round_half(O):
    """binary16 rounding (ties to even) equals numpy's float16 conversion, subnormals and overflow included."""
    rng = np.random.default_rng(3)
    vals = np.concatenate([
        rng.standard_normal(3000).astype(np.float32) * np.float32(3.0),
        (rng.standard_normal(1000) * 1e-5).astype(np.float32),           # binary16 subnormals
        (rng.standard_normal(500) * 3e4).astype(np.float32),              # near overflow
        np.array([65504.0, 65519.99, 65520.0, -65520.0, 2.0 ** -24, 2.0 ** -25, 3 * 2.0 ** -26,
                  1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11, -0.0, 0.0], dtype=np.float32)])
    # exact ties between neighbouring binary16 values
    h = rng.standard_normal(500).astype(np.float16)
    nxt = np.nextafter(h, np.float16(np.inf))
    ties = ((h.astype(np.float64) + nxt.astype(np.float64)) / 2).astype(np.float32)
    vals = np.concatenate([vals, ties])
    for v in vals:
        got = O.round_half(float(v))
        with np.errstate(over="ignore"):
            want = float(np.float32(v).astype(np.float16))
        assert (got == want) or (np.isnan(got) and np.isnan(want)), f"round_half({v!r}) = {got}, numpy {want}"
        assert np.signbit(got) == np.signbit(want)


def pin_metric_f16(O):
    """The binary16 inversion function equals numpy's float16 arithmetic on the same operands."""
    rng = np.random.default_rng(6)
    for _ in range(3000):
        y16 = np.float16(rng.normal() * 1.5)
        w16 = np.float16(rng.uniform(0.05, 1.5))
        S = int(rng.integers(-7, 8))
        x = int(rng.choice([-1, 1]))
        q = np.float32(rng.normal() * 0.7)
        xy = y16 if x > 0 else -y16
        want = np.float16(np.float16(xy + np.float16(w16 * np.float16(S))) + np.float16(q))
        got = O.metric_f16(x, float(y16), S, float(w16), float(q))
        assert got == float(want), (x, y16, S, w16, q, got, want)


def pin_metric_f32_f64(O):
    """E_k = ((x_k y_k) + w S_k) + q_k with one rounding per operation, in this order: FP32 equals
    numpy float32 arithmetic and FP64 numpy float64 arithmetic on the same operands."""
    rng = np.random.default_rng(7)
    for _ in range(3000):
        ys = np.float32(rng.normal() * 1.5)
        w = np.float32(rng.uniform(0.0, 1.5))
        S = int(rng.integers(-7, 8))
        x = int(rng.choice([-1, 1]))
        q = np.float32(rng.normal() * 0.7)
        xy = ys if x > 0 else -ys
        want = (xy + w * np.float32(S)) + q
        assert np.float32(O.metric_f32(x, float(ys), S, float(w), float(q))) == want
        want64 = (float(xy) + float(w) * S) + float(q)
        assert O.metric_f64(x, float(ys), S, float(w), float(q)) == want64


def pin_fix_quantizer(O):
    """The FP32-decided level code agrees with Eq. 8 (g in double) away from level boundaries;
    saturation, the missing zero level and the sign convention hold."""
    rng = np.random.default_rng(4)
    for q_bits, y_max in ((3, 2.5), (4, 1.5), (5, 1.75), (8, 2.5), (8, 2.0)):
        R = O.fix_scale(q_bits, y_max)
        assert R == float(np.float32(2.0 ** q_bits / (2.0 * np.float32(y_max))))
        kmax = 2 ** (q_bits - 1) - 1
        d = 2.0 * y_max / 2 ** q_bits
        for v in rng.uniform(-1.3 * y_max, 1.3 * y_max, 2000).astype(np.float32):
            frac = abs(float(v)) / d
            if abs(frac - round(frac)) < 1e-4:
                continue                       # FP32 and FP64 may decide a boundary differently
            b = O.fix_code(float(v), R, kmax)
            assert -kmax - 1 <= b <= kmax
            assert (2 * b + 1) * d / 2 == O.quantize(float(v), q_bits, y_max)
        assert O.fix_code(0.0, R, kmax) == 0 and O.fix_code(-0.0, R, kmax) == 0
        assert O.fix_code(1e30, R, kmax) == kmax and O.fix_code(-1e30, R, kmax) == -kmax - 1


def pin_table2_fixed_point(O):
    """Table II again, through the decoder's fixed-point thresholds Theta~(u) = V(fl32(theta lambda^u))."""
    want = {}
    for q, i, th, tau in _golden_lines("table2_threshold_events.txt"):
        want.setdefault(int(q), []).append((float(th), int(tau)))
    thr = O.threshold_table_f32(-0.9, 0.99, 300)
    for q, events in want.items():
        R = O.fix_scale(q, 2.5)
        kmax = 2 ** (q - 1) - 1
        d = 5.0 / 2 ** q
        vals = [(2 * O.fix_code(float(t), R, kmax) + 1) * d / 2 for t in thr]
        got = [(vals[0], 0)] + [(vals[u], u) for u in range(1, len(vals)) if vals[u] != vals[u - 1]]
        assert [(round(a, 4), b) for a, b in got] == events, (q, got)


def pin_trace_fixed_point(O):
    """Case I (Q = 4, Y_max = 2, Delta = 1/4, levels in units of Delta/2): y = (3,3,3,-3,3,3,3)
    saturates to Y~ = (15,15,15,-15,15,15,15); w = 0.875 -> W~ = 7; theta = -0.375 -> Theta~ = -3;
    eta = 0 -> q~ = V(0) = +1.  At t = 0 all three checks fail: E~_3 = 15 + 7(-3) + 1 = -5 < -3
    flips x_3; E~_0,1,2 = 15 - 14 + 1 = 2 and E~_4,5,6 = 15 - 7 + 1 = 9 do not.  t = 1 is valid."""
    C = hamming_code()
    y = np.array([3, 3, 3, -3, 3, 3, 3], np.float32)
    p = oracle_pkg.make_params(w=0.875, theta=-0.375, eta=0.0, lam=1.0, y_max=2.0, t_max=6,
                               precision=oracle_pkg.FIX, q_bits=4)
    bits, it, ps = O.decode_f32(C, y[None, :], 0.5, p, seed=1)
    assert (int(bits[0, 0]), int(it[0]), int(ps[0])) == (0, 1, 1)
    # theta = -0.625 -> Theta~ = -5: E~_3 = -5 is a tie, nothing flips, T is reached
    p = oracle_pkg.make_params(w=0.875, theta=-0.625, eta=0.0, lam=1.0, y_max=2.0, t_max=6,
                               precision=oracle_pkg.FIX, q_bits=4)
    bits, it, ps = O.decode_f32(C, y[None, :], 0.5, p, seed=1)
    assert (int(bits[0, 0]), int(it[0]), int(ps[0])) == (0x08, 6, 0)


def _dyadic_frames(C, F, step, seed):
    rng = np.random.default_rng(seed)
    y, cw, _ = wl.frames(C, F, None, seed=seed)
    noise = rng.integers(-16, 17, size=y.shape) * step
    return (y + noise).astype(np.float32)


def pin_fp16_reduces_to_fp32(O):
    """With eta = 0 and inputs on a coarse dyadic grid every FP32 intermediate is a binary16
    value, so the FP16 decoder must equal the FP32 decoder exactly."""
    C = _pin_code()
    y = _dyadic_frames(C, 40, 1.0 / 16, seed=21)
    for variant in (0, 2):
        p32 = oracle_pkg.make_params(w=0.5, theta=-0.75, eta=0.0, lam=1.0, t_max=30, smooth_window=8,
                                     variant=variant, precision=oracle_pkg.FP32)
        p16 = oracle_pkg.make_params(w=0.5, theta=-0.75, eta=0.0, lam=1.0, t_max=30, smooth_window=8,
                                     variant=variant, precision=oracle_pkg.FP16)
        a = O.decode_f32(C, y, 0.5, p32, seed=1)
        b = O.decode_f32(C, y, 0.5, p16, seed=1)
        assert all((u == v).all() for u, v in zip(a, b))
        assert (a[2] == 0).any() and (a[2] == 1).any()


def pin_fix_reduces_to_fp32(O):
    """With Q = 4, Y_max = 2 (Delta = 1/4) and y, w, theta at level centres, eta = 0 gives
    q~ = V(0) = +1, i.e. E~ (Delta/2) = E + Delta/2: the fixed-point decoder must equal the FP32
    decoder run with theta - Delta/2."""
    C = _pin_code()
    rng = np.random.default_rng(22)
    y, _, _ = wl.frames(C, 40, None, seed=22)
    centres = (2 * rng.integers(-8, 8, size=y.shape) + 1) * 0.125   # +-0.125 .. +-1.875
    y = np.where(y > 0, np.abs(centres), -np.abs(centres)).astype(np.float32)
    # saturated samples: the fixed-point level tops out at 15 * Delta/2 = 1.875, which the FP32
    # run reproduces by clamping at 1.875
    y = np.where(rng.random(y.shape) < 0.25, np.sign(y) * 3.0, y).astype(np.float32)
    y = np.where(rng.random(y.shape) < 0.02, -y, y).astype(np.float32)    # errors to correct
    for variant in (0, 2):
        pfix = oracle_pkg.make_params(w=0.375, theta=-0.625, eta=0.0, lam=1.0, y_max=2.0, t_max=30,
                                      smooth_window=8, variant=variant, precision=oracle_pkg.FIX, q_bits=4)
        p32 = oracle_pkg.make_params(w=0.375, theta=-0.75, eta=0.0, lam=1.0, y_max=1.875, t_max=30,
                                     smooth_window=8, variant=variant, precision=oracle_pkg.FP32)
        a = O.decode_f32(C, y, 0.5, pfix, seed=1)
        b = O.decode_f32(C, y, 0.5, p32, seed=1)
        assert all((u == v).all() for u, v in zip(a, b))
        assert (a[2] == 0).any() and (a[2] == 1).any()


def pin_precision_statistics(O):
    """FP16 and 8-bit fixed point decode the same frames to nearly the FP32 results."""
    C = _pin_code()
    y, _, sig = wl.frames(C, 300, 3.0, seed=23)
    res = {}
    for prec, qb in ((oracle_pkg.FP32, 0), (oracle_pkg.FP16, 0), (oracle_pkg.FIX, 8)):
        p = oracle_pkg.make_params(w=0.75, theta=-0.9, eta=0.9, lam=0.95, t_max=50, variant=3,
                                   precision=prec, q_bits=qb)
        res[prec] = O.decode_f32(C, y, sig, p, seed=2)
    for prec in (oracle_pkg.FP16, oracle_pkg.FIX):
        assert abs(res[prec][2].mean() - res[oracle_pkg.FP32][2].mean()) < 0.06
        assert (res[prec][1] == res[oracle_pkg.FP32][1]).mean() > 0.3


# ---------------------------------------------------------------------------
# uniform perturbation (Sec. V-B), accumulating fixed point, objective trace
# ---------------------------------------------------------------------------

def pin_uniform_deviate(O):
    """v(r) = (2 (r >> 8) + 1 - 2^24) 2^-24: closed forms at the ends and the middle, odd multiples
    of 2^-24, exact symmetry v(~r) = -v(r), and the uniform law on (-1, 1) with variance 1/3."""
    from scipy import stats
    two24 = 2.0 ** -24
    for r, want in ((0, -1.0 + two24), (0xFFFFFFFF, 1.0 - two24), (0x80000000, two24),
                    (0x7FFFFFFF, -two24), (0x800000FF, two24), (0x00000100, -1.0 + 3 * two24)):
        assert float(O.uniform_f32(r)) == want, (hex(r), float(O.uniform_f32(r)), want)
    rng = np.random.default_rng(31)
    r = rng.integers(0, 2 ** 32, size=20000, dtype=np.uint64)
    v = np.array([float(O.uniform_f32(int(x))) for x in r])
    odd = v * 2 ** 24
    assert (odd == np.round(odd)).all() and (np.mod(np.round(odd), 2) == 1).all()
    assert all(float(O.uniform_f32(int(x) ^ 0xFFFFFFFF)) == -vv for x, vv in zip(r[:2000], v[:2000]))
    assert stats.kstest(v, "uniform", args=(-1.0, 2.0)).pvalue > 1e-4
    assert abs(v.mean()) < 0.02 and abs(v.var() - 1.0 / 3.0) < 0.01


def pin_uniform4_wiring(O):
    """Uniform deviate of symbol 4g + i = output i of Philox counter (g, t, frame_lo, frame_hi)."""
    for seed, f, t, g in ((12345, 0, 0, 0), (7, 3, 299, 511), ((5 << 32) | 9, (2 << 32) | 1, 17, 3)):
        r = O.philox([g, t, f & 0xFFFFFFFF, f >> 32], [seed & 0xFFFFFFFF, seed >> 32])
        v = O.uniform4_f32(seed, f, t, g)
        for i in range(4):
            assert v[i] == O.uniform_f32(int(r[i]))


def pin_uniform_noise_in_decoder(O):
    """With the UNIFORM variant bit the FP32 decoder adds q_k = fl32(eta sigma sqrt 3) v_k each
    iteration (variance eta^2 sigma^2, the Gaussian's), with v_k from the same Philox counter."""
    C = _pin_code()
    y, _, sig = wl.frames(C, 6, 1.0, seed=13)
    eta = 0.96
    scale = np.float32(float(np.float32(eta)) * float(np.float32(sig)) * math.sqrt(3.0))
    assert abs(float(scale) / math.sqrt(3.0) - eta * sig) < 1e-6
    for variant in (oracle_pkg.UNIFORM, oracle_pkg.UNIFORM | 3):
        p = oracle_pkg.make_params(w=0.75, theta=-0.9, eta=eta, lam=0.97, t_max=25, smooth_window=9,
                                   variant=variant)
        b2, it2, ps2 = O.decode_f32(C, y, sig, p, seed=5, frame_offset=40)
        for f in range(6):
            v = np.array([np.concatenate([O.uniform4_f32(5, 40 + f, t, g) for g in range(C.n // 4)])
                          for t in range(25)], np.float32)
            q = (scale * v).astype(np.float32)
            b1, it1, ps1 = O.decode_f32_qin(C, y[f], p, q)
            assert (b1 == b2[f]).all() and it1 == it2[f] and ps1 == ps2[f], f"frame {f}"
        # the Gaussian decoder on the same frames takes other decisions (the bit is honoured)
        pg = oracle_pkg.make_params(w=0.75, theta=-0.9, eta=eta, lam=0.97, t_max=25, smooth_window=9,
                                    variant=variant & ~oracle_pkg.UNIFORM)
        bg, itg, _ = O.decode_f32(C, y, sig, pg, seed=5, frame_offset=40)
        assert not ((bg == b2).all() and (itg == it2).all())


def pin_fixacc_scale_and_steps(O):
    """Rd = fl32(2^(Q+8) / Y_max) and steps(v) = rint(fl32(v Rd)) (ties to even)."""
    assert O.fixacc_scale(8, 2.5) == float(np.float32(65536 / 2.5))
    assert O.fixacc_scale(4, 2.0) == 2048.0
    R = O.fixacc_scale(8, 2.5)
    assert O.fixacc_steps(0.75, R) == 19661          # 19660.8
    assert O.fixacc_steps(-0.9, R) == -23593         # -23592.96
    assert O.fixacc_steps(0.5 / 2048, 2048.0) == 0   # 0.5 ties to even
    assert O.fixacc_steps(1.5 / 2048, 2048.0) == 2   # 1.5 ties to even
    assert O.fixacc_steps(-0.0003, 2048.0) == -1     # -0.6144


def pin_trace_fixacc(O):
    """Case K (Q = 4, Y_max = 2: Rd = 2048 steps per unit, 256 per half level of Delta/2 = 1/8):
    y = (3,3,3,-3,3,3,3) holds level codes (7,7,7,-8,7,7,7), i.e. +-15 half levels = +-3840 steps;
    w = 0.875 -> W = 1792; theta = -0.375 -> Theta = -768.  t = 0: s = (-1,-1,-1), E_3 =
    3840 - 3 * 1792 = -1536 < -768 flips x_3; E_0,1,2 = 3840 - 3584 = 256 and E_4,5,6 = 2048 do not;
    t = 1 is valid.  theta = -0.75 (Theta = -1536) makes E_3 a tie: nothing flips (T reached); an
    injected q_3(0) = -0.0003 (-1 step) breaks the tie and x_3 flips, q_3(0) = +0.3 (614 steps) does not."""
    C = hamming_code()
    y = np.array([3, 3, 3, -3, 3, 3, 3], np.float32)

    def run(theta, q3=None):
        p = oracle_pkg.make_params(w=0.875, theta=theta, eta=0.0, lam=1.0, y_max=2.0, t_max=6,
                                   precision=oracle_pkg.FIXACC, q_bits=4)
        if q3 is None:
            bits, it, ps = O.decode_f32(C, y[None, :], 0.5, p, seed=1)
            return int(bits[0, 0]), int(it[0]), int(ps[0])
        q = np.zeros((6, 7), np.float32)
        q[0, 3] = q3
        bits, it, ps = O.decode_f32_qin(C, y, p, q)
        return _bits_byte(bits), it, ps
    assert run(-0.375) == (0, 1, 1)
    assert run(-0.75) == (0x08, 6, 0)
    assert run(-0.75, -0.0003) == (0, 1, 1)
    assert run(-0.75, 0.3) == (0x08, 6, 0)


def _eq8_value(y, q_bits, y_max):
    """g(y) of Eq. 8 with the saturating level index, in double (the level decided in FP32)."""
    nq = 2 ** q_bits
    a = np.abs(np.asarray(y, np.float32)) * np.float32(nq / (2.0 * y_max))
    k = np.minimum(np.floor(a), nq // 2 - 1)
    return np.where(np.asarray(y) >= 0, 1.0, -1.0) * (k + 0.5) * (2.0 * y_max / nq)


def pin_fixacc_is_exact_on_its_grid(O):
    """When w, theta and every perturbation are multiples of the accumulator step (Y_max = 2, Q = 8:
    step 2^-15), the accumulating fixed point takes exactly the real-arithmetic decisions on the
    quantized samples g(y): it equals the FP32 decoder fed g(y), whose sums are then exact."""
    C = _pin_code()
    y, _, sig = wl.frames(C, 8, 2.0, seed=24)
    T = 30
    rng = np.random.default_rng(25)
    gy = _eq8_value(y, 8, 2.0).astype(np.float32)
    for variant in (0, oracle_pkg.SMOOTH):
        pacc = oracle_pkg.make_params(w=0.75, theta=-0.875, eta=0.0, lam=1.0, y_max=2.0, t_max=T,
                                      smooth_window=8, variant=variant, precision=oracle_pkg.FIXACC, q_bits=8)
        p32 = oracle_pkg.make_params(w=0.75, theta=-0.875, eta=0.0, lam=1.0, y_max=2.0, t_max=T,
                                     smooth_window=8, variant=variant, precision=oracle_pkg.FP32)
        passes = []
        for f in range(y.shape[0]):
            q = (np.round(rng.normal(0, 0.5, size=(T, C.n)) * 2 ** 15) / 2 ** 15).astype(np.float32)
            a = O.decode_f32_qin(C, y[f], pacc, q)
            b = O.decode_f32_qin(C, gy[f], p32, q)
            assert (a[0] == b[0]).all() and a[1:] == b[1:], f"frame {f}"
            passes.append(a[2])
        assert 0 < sum(passes) < len(passes)


def pin_fixacc_statistics(O):
    """The 8-bit accumulating fixed point decodes the same frames almost always as FP32 does
    (only the held sample is quantized; E keeps 2^-16 resolution relative to Y_max)."""
    C = _pin_code()
    y, _, sig = wl.frames(C, 300, 3.0, seed=23)
    res = {}
    for prec, qb in ((oracle_pkg.FP32, 0), (oracle_pkg.FIXACC, 8)):
        p = oracle_pkg.make_params(w=0.75, theta=-0.9, eta=0.9, lam=0.95, t_max=50, variant=3,
                                   precision=prec, q_bits=qb)
        res[prec] = O.decode_f32(C, y, sig, p, seed=2)
    assert abs(res[oracle_pkg.FIXACC][2].mean() - res[oracle_pkg.FP32][2].mean()) < 0.05
    assert (res[oracle_pkg.FIXACC][1] == res[oracle_pkg.FP32][1]).mean() > 0.3


def _dense_syndrome_weight(H, x):
    return int(((H.astype(np.int64) @ (x < 0).astype(np.int64)) % 2).sum())


def _corr_fixed(x, yv):
    """sum_k rint(x_k y_k 2^32) in exact integers (numpy's rint: ties to even)."""
    return int(np.rint(np.ldexp(x * np.asarray(yv, np.float64), 32)).astype(np.int64).sum())


def pin_objective_trace(O):
    """Objective trace f(x(t)) = C(t) 2^-32 + m - 2 U(t) (Sec. III-B objective):
    - t = 0: x(0) = sign(y~), so U(0) is the syndrome weight of sign(y~) (dense H) and
      C(0) = sum rint(|y~_k| 2^32), for FP32, FP64 and the Eq. 8 held samples;
    - at t = iters of a passing frame, U = 0 and C is the correlation of the output word;
    - entries after iters are not written;
    - eta = 0, lambda = 1: the whole trace equals textbook M-GDBF's f(x(t)) evaluated densely."""
    C = _pin_code()
    H = C.dense()
    y, _, sig = wl.frames(C, 24, 2.5, seed=26)
    yc = np.clip(y, -2.5, 2.5)
    T = 40
    cases = [("f32", oracle_pkg.FP32, 0, yc), ("fix", oracle_pkg.FIX, 6, _eq8_value(yc, 6, 2.5)),
             ("acc", oracle_pkg.FIXACC, 8, _eq8_value(yc, 8, 2.5))]
    for name, prec, qb, held in cases:
        p = oracle_pkg.make_params(w=0.75, theta=-0.9, eta=0.9, lam=0.97, y_max=2.5, t_max=T, variant=1,
                                   precision=prec, q_bits=qb)
        for arith in ("f32", "f64"):
            if arith == "f64" and prec != oracle_pkg.FP32:
                continue                      # the FP64 decoder holds unquantized samples
            dec = O.decode_f64_trace if arith == "f64" else O.decode_f32_trace
            bits, it, ps, tu, tc = dec(C, y, sig, p, 20, seed=3)
            out = 1 - 2 * wl.unpack_bits(bits, C.n).astype(np.int64)
            for f in range(20):
                x0 = np.where(held[f] >= 0, 1, -1)
                assert tu[f, 0] == _dense_syndrome_weight(H, x0), (name, f)
                assert tc[f, 0] == _corr_fixed(np.ones(C.n), np.abs(held[f])), (name, f)
                assert (tu[f, it[f] + 1:] == -1).all() and (tc[f, it[f] + 1:] == 0).all()
                assert (tu[f, :it[f] + 1] >= 0).all()
                if ps[f]:
                    assert tu[f, it[f]] == 0 and tc[f, it[f]] == _corr_fixed(out[f], held[f]), (name, f)
                else:
                    assert tu[f, it[f]] > 0 and tc[f, it[f]] == _corr_fixed(out[f], held[f]), (name, f)
            assert (ps == 1).any() and (ps == 0).any() and (it > 2).any()
    # eta = 0: dense M-GDBF objective trajectory
    p = oracle_pkg.make_params(w=0.75, theta=-0.9, eta=0.0, lam=1.0, y_max=2.5, t_max=T, variant=0)
    bits, it, ps, tu, tc = O.decode_f64_trace(C, y, sig, p, 24, seed=3)
    Hi = H.astype(np.int64)
    w, th = float(np.float32(0.75)), float(np.float32(-0.9))
    for f in range(24):
        x = np.where(yc[f] >= 0, 1, -1)
        for t in range(it[f] + 1):
            U = _dense_syndrome_weight(H, x)
            assert tu[f, t] == U, (f, t)
            assert abs(tc[f, t] * 2.0 ** -32 - float(x @ yc[f].astype(np.float64))) <= C.n * 2.0 ** -33
            s = 1 - 2 * ((Hi @ (x < 0).astype(np.int64)) % 2)
            E = x * yc[f].astype(np.float64) + w * (Hi.T @ s)
            x = np.where(E < th, -x, x)


ALL_PINS = [
    pin_philox_kat, pin_icdf_vs_library, pin_icdf_symmetry_and_range, pin_gauss_f64_vs_library,
    pin_gauss4_wiring, pin_gauss_statistics,
    pin_noise_variance, pin_threshold_table, pin_table2, pin_fig20, pin_quantizer,
    pin_trace_gdbf, pin_trace_injected_noise, pin_trace_adaptation, pin_trace_smoothing,
    pin_trace_clamp_sign_tie, pin_trace_single_bit, pin_noiseless, pin_eta0_is_gdbf,
    pin_eta0_is_single_bit_gdbf, pin_codeword_and_ml,
    pin_f32_matches_injected_noise, pin_frame_independence, pin_f32_f64_statistics,
    pin_round_half, pin_metric_f16, pin_metric_f32_f64, pin_fix_quantizer, pin_trace_fixed_point, pin_table2_fixed_point, pin_fp16_reduces_to_fp32,
    pin_fix_reduces_to_fp32, pin_precision_statistics,
    pin_uniform_deviate, pin_uniform4_wiring, pin_uniform_noise_in_decoder, pin_fixacc_scale_and_steps,
    pin_trace_fixacc, pin_fixacc_is_exact_on_its_grid, pin_fixacc_statistics, pin_objective_trace,
]
