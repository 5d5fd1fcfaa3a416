"""Objective function and convergence error (Sec. III-B Eq. 2, Sec. VI Eqs. 17-18)."""
import numpy as np

import oracle
from paper_1402_2773_gb300 import diagnostics as dg, workload as wl


def test_codewords_satisfy_every_check_and_reach_f_max():
    """Sum of s_i = m for a codeword (Sec. III-B); f(c^) = sum c^ y + m = f_max (Sec. VI)."""
    code = wl.code_c1()
    y, cw, _ = wl.frames(code, 50, 3.0, seed=2)
    x = dg.bipolar(cw, code.n)
    assert (dg.syndrome_sum(code, x) == code.m).all()
    assert np.allclose(dg.objective(code, y, cw), dg.f_max(code, y, cw))
    assert dg.convergence_error(code, y, cw, cw) == 0.0


def test_syndrome_sum_against_dense_parity():
    code = wl.peg_code(96, 48, 3, seed=11)
    rng = np.random.default_rng(1)
    bits = np.packbits(rng.integers(0, 2, (40, 96)).astype(np.uint8), axis=1, bitorder="little")
    x = dg.bipolar(bits, 96)
    H = code.dense().astype(np.int64)
    s = 1 - 2 * (((x < 0).astype(np.int64) @ H.T) % 2)
    assert (dg.syndrome_sum(code, x) == s.sum(axis=1)).all()


def test_convergence_error_orders_decoders_as_the_paper_reports():
    """Sec. VI (Fig. 18, 5 dB, T = 100): the noisy decoders end closer to the global maximum than
    M-GDBF; every passing frame has f = its codeword's correlation + m."""
    O = oracle.load()
    code = wl.code_c1()
    y, cw, sig = wl.frames(code, 200, 5.0, seed=3)
    eps = {}
    for name, variant, eta, lam in (("M-GDBF", 0, 0.0, 1.0), ("M-NGDBF", 0, 0.96, 1.0),
                                    ("AT-NGDBF", 1, 0.96, 0.99)):
        p = oracle.make_params(w=0.75, theta=-0.9, eta=eta, lam=lam, t_max=100, variant=variant)
        bits, it, ps = O.decode_f32(code, y, sig, p, seed=4, threads=8)
        eps[name] = dg.convergence_error(code, y, bits, cw, y_max=2.5)
        f = dg.objective(code, y, bits, y_max=2.5)
        corr = (dg.bipolar(bits, code.n) * np.clip(y, -2.5, 2.5)).sum(axis=1)
        assert np.allclose(f[ps == 1], corr[ps == 1] + code.m)
    assert eps["M-NGDBF"] > eps["M-GDBF"] and eps["AT-NGDBF"] > eps["M-GDBF"]
    assert eps["AT-NGDBF"] >= eps["M-NGDBF"] - 1e-9
