"""CUDA decoder vs the reference decoder for the uniform perturbation (Sec. V-B), the accumulating
8-bit fixed point (Sec. IV-E) and the objective trace (Sec. III-B objective, Sec. VI).

Bits, iteration counts, pass flags and every trace entry are compared exactly, through the C ABI.
The convergence error of Sec. VI is then evaluated from the GPU's own outputs.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1402_2773_gb300 import diagnostics as dg, ngdbf, workload as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1
U = ngdbf.NGDBF_UNIFORM


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_2773_gb300 import _build
    _build.build_cuda()
    ngdbf.load()
    torch.cuda.set_device(0)


@pytest.fixture(scope="module")
def O():
    return oracle.load()


def params_pair(**kw):
    d = dict(w=0.75, theta=-0.9, eta=0.96, lam=1.0, y_max=2.5, t_max=100, smooth_window=64, variant=0,
             precision=ngdbf.NGDBF_FP32, q_bits=0)
    d.update(kw)
    return ngdbf.make_params(**d), oracle.make_params(**d)


def gpu_decode(code, y, sigma, gp, seed, frame_offset=0):
    dc = ngdbf.DeviceCode.from_code(code)
    try:
        yt = torch.from_numpy(np.ascontiguousarray(y)).cuda()
        b, i, p = dc.decode(yt, sigma, gp, seed=seed, frame_offset=frame_offset)
        torch.cuda.synchronize()
        return b.cpu().numpy(), i.cpu().numpy(), p.cpu().numpy()
    finally:
        dc.close()


def assert_parity(O, code, y, sigma, seed=1, frame_offset=0, **kw):
    gp, op = params_pair(**kw)
    gb, gi, gps = gpu_decode(code, y, sigma, gp, seed, frame_offset)
    ob, oi, ops = O.decode_f32(code, y, sigma, op, seed=seed, frame_offset=frame_offset, threads=THREADS)
    bad = np.nonzero((gb != ob).any(axis=1) | (gi != oi) | (gps != ops))[0]
    assert bad.size == 0, f"{bad.size}/{y.shape[0]} frames differ, first {bad[:5]}"
    return gb, oi, ops


PRECS = {"fp32": (ngdbf.NGDBF_FP32, 0), "fp16": (ngdbf.NGDBF_FP16, 0), "fix6": (ngdbf.NGDBF_FIX, 6),
         "acc8": (ngdbf.NGDBF_FIXACC, 8), "acc4": (ngdbf.NGDBF_FIXACC, 4)}


@pytest.mark.parametrize("variant", [U, U | 1, U | 2, U | 3, U | 4, U | 6])
@pytest.mark.parametrize("prec", ["fp32", "fix6", "acc8"])
def test_uniform_perturbation(O, variant, prec):
    code = wl.peg_code(96, 48, 3, seed=11)
    y, _, sig = wl.frames(code, 130, 2.5, seed=41)
    p, qb = PRECS[prec]
    lam = 1.0 if variant & 4 else 0.95
    _, it, ps = assert_parity(O, code, y, sig, seed=9, frame_offset=77, variant=variant, lam=lam, t_max=60,
                              smooth_window=16, precision=p, q_bits=qb)
    assert (ps == 0).any() and (ps == 1).any()


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 6])
@pytest.mark.parametrize("prec", ["acc8", "acc4"])
def test_fixacc_small(O, variant, prec):
    code = wl.peg_code(96, 48, 3, seed=11)
    y, _, sig = wl.frames(code, 100, 2.5, seed=4)
    p, qb = PRECS[prec]
    lam = 1.0 if variant & 4 else 0.95
    assert_parity(O, code, y, sig, seed=9, variant=variant, lam=lam, t_max=60, smooth_window=16,
                  precision=p, q_bits=qb)


def test_fixacc_workloads(O):
    """(3,6) N=1008 plain and (6,32) N=2048 SM-NGDBF, 8-bit held samples."""
    code = wl.code_c1()
    y, _, sig = wl.frames(code, 1500, 4.0, seed=42)
    assert_parity(O, code, y, sig, seed=1, w=0.75, theta=-0.9, eta=0.96, t_max=100,
                  precision=ngdbf.NGDBF_FIXACC, q_bits=8)
    code = wl.code_c2()
    y, _, sig = wl.frames(code, 200, 3.75, seed=43)
    assert_parity(O, code, y, sig, seed=7, w=0.1875, theta=-0.7, eta=0.65, lam=0.993, y_max=2.0, t_max=300,
                  smooth_window=64, variant=3, precision=ngdbf.NGDBF_FIXACC, q_bits=8)


def test_fixacc_global_state_and_wide(O):
    """Per-slot state in global memory (N = 8192) and bit-sliced counts (symbol degree 9)."""
    code = wl.peg_code(8192, 1639, 3, seed=1)
    y, _, sig = wl.frames(code, 64, 3.0, seed=44)
    assert_parity(O, code, y, sig, seed=2, lam=0.97, t_max=40, smooth_window=10, variant=3,
                  precision=ngdbf.NGDBF_FIXACC, q_bits=8)
    assert ngdbf.ngdbf_last_launch()["state_in_smem"] == 0
    code = wl.peg_code(360, 120, 9, seed=3)
    y, _, sig = wl.frames(code, 70, 3.0, seed=45)
    assert_parity(O, code, y, sig, seed=3, w=0.3, theta=-0.6, eta=0.7, lam=0.97, t_max=50, variant=3 | U,
                  smooth_window=12, precision=ngdbf.NGDBF_FIXACC, q_bits=8)


def test_fixacc_range_is_checked():
    code = wl.peg_code(96, 48, 3, seed=11)
    dc = ngdbf.DeviceCode.from_code(code)
    try:
        y = torch.zeros((4, 96), dtype=torch.float32, device="cuda")
        gp = ngdbf.make_params(w=0.75, theta=-0.9, eta=1.0, y_max=2.5, t_max=10, precision=ngdbf.NGDBF_FIXACC,
                               q_bits=8)
        with pytest.raises(ngdbf.NgdbfError) as e:
            dc.decode(y, 1e5, gp)             # 8 sigma = 8e5 units, beyond 2^28 steps
        assert e.value.status == ngdbf.NGDBF_ERR_UNSUPPORTED
    finally:
        dc.close()


def trace_pair(O, code, y, sigma, K, seed=3, frame_offset=0, **kw):
    gp, op = params_pair(**kw)
    dc = ngdbf.DeviceCode.from_code(code)
    try:
        yt = torch.from_numpy(np.ascontiguousarray(y)).cuda()
        gb, gi, gps, gu, gc = [t.cpu().numpy() for t in dc.decode_trace(yt, sigma, gp, K, seed=seed,
                                                                        frame_offset=frame_offset)]
        torch.cuda.synchronize()
    finally:
        dc.close()
    ob, oi, ops, ou, oc = O.decode_f32_trace(code, y, sigma, op, K, seed=seed, frame_offset=frame_offset,
                                             threads=THREADS)
    assert np.array_equal(gb, ob) and np.array_equal(gi, oi) and np.array_equal(gps, ops)
    for f in range(K):
        L = oi[f] + 1
        assert np.array_equal(gu[f, :L], ou[f, :L]), f"frame {f}: U(t) differs"
        assert np.array_equal(gc[f, :L], oc[f, :L]), f"frame {f}: C(t) differs"
    return gb, gi, gps, gu, gc


@pytest.mark.parametrize("variant,prec", [(0, "fp32"), (3, "fp32"), (3, "fp16"), (1, "fix6"), (3, "acc8"),
                                          (4, "fp32"), (6 | U, "fp32"), (3 | U, "acc8")])
def test_objective_trace(O, variant, prec):
    """U(t) and C(t) of 150 traced frames (of 230, spread over several CTAs and slot refills)."""
    code = wl.peg_code(96, 48, 3, seed=11)
    y, _, sig = wl.frames(code, 230, 2.5, seed=46)
    p, qb = PRECS[prec]
    lam = 1.0 if variant & 4 else 0.95
    gb, gi, gps, gu, gc = trace_pair(O, code, y, sig, 150, frame_offset=500, variant=variant, lam=lam, t_max=60,
                                     smooth_window=16, precision=p, q_bits=qb)
    assert (gi[:150] > 3).sum() > 20
    # the last entry of a passing frame: no unsatisfied check, the correlation of its output
    f = dg.objective(code, y, gb, y_max=2.5) if prec in ("fp32",) else None
    for k in range(150):
        if gps[k]:
            assert gu[k, gi[k]] == 0
            if f is not None:
                assert abs(gc[k, gi[k]] * 2.0 ** -32 + code.m - f[k]) <= code.n * 2.0 ** -33 + 1e-9


def test_objective_trace_workload(O):
    """(6,32) N=2048 SM-NGDBF at 3.75 dB, trace of 64 frames over T = 300."""
    code = wl.code_c2()
    y, _, sig = wl.frames(code, 96, 3.75, seed=47)
    trace_pair(O, code, y, sig, 64, seed=7, w=0.1875, theta=-0.7, eta=0.65, lam=0.993, y_max=2.0, t_max=300,
               smooth_window=64, variant=3)


def test_trace_arguments():
    code = wl.peg_code(96, 48, 3, seed=11)
    dc = ngdbf.DeviceCode.from_code(code)
    try:
        y = torch.zeros((4, 96), dtype=torch.float32, device="cuda")
        gp = ngdbf.make_params(t_max=10)
        b = torch.empty((4, 12), dtype=torch.uint8, device="cuda")
        i = torch.empty(4, dtype=torch.int32, device="cuda")
        p = torch.empty(4, dtype=torch.uint8, device="cuda")
        tu = torch.empty((4, 11), dtype=torch.int32, device="cuda")
        tc = torch.empty((4, 11), dtype=torch.int64, device="cuda")
        s = torch.cuda.current_stream().cuda_stream
        args = (dc.handle, y.data_ptr(), 4, 0.5, gp, 1, 0, b.data_ptr(), i.data_ptr(), p.data_ptr())
        for K, u_ptr, c_ptr in ((5, tu.data_ptr(), tc.data_ptr()), (-1, tu.data_ptr(), tc.data_ptr()),
                                (2, 0, tc.data_ptr()), (2, tu.cpu().data_ptr(), tc.data_ptr())):
            with pytest.raises(ngdbf.NgdbfError) as e:
                ngdbf.ngdbf_decode_trace(*args, K, u_ptr, c_ptr, s)
            assert e.value.status == ngdbf.NGDBF_ERR_INVALID_ARG
        gp0 = ngdbf.make_params(t_max=10, y_max=0.0)
        with pytest.raises(ngdbf.NgdbfError):
            ngdbf.ngdbf_decode_trace(dc.handle, y.data_ptr(), 4, 0.5, gp0, 1, 0, b.data_ptr(), i.data_ptr(),
                                     p.data_ptr(), 2, tu.data_ptr(), tc.data_ptr(), s)
        ngdbf.ngdbf_decode_trace(*args, 0, 0, 0, s)           # no trace: a plain decode
        torch.cuda.synchronize()
    finally:
        dc.close()


def test_convergence_error_from_gpu_outputs(O):
    """Sec. VI (Eqs. 17-18) on the GPU's own outputs: the convergence error equals the reference
    decoder's, and the noisy decoders end closer to the global maximum than M-GDBF."""
    code = wl.code_c1()
    y, cw, sig = wl.frames(code, 400, 5.0, seed=3)
    eps = {}
    for name, variant, eta, lam in (("M-GDBF", 0, 0.0, 1.0), ("M-NGDBF", 0, 0.96, 1.0),
                                    ("AT-NGDBF", 1, 0.96, 0.99), ("M-NGDBF uniform", U, 0.96, 1.0)):
        gp, op = params_pair(w=0.75, theta=-0.9, eta=eta, lam=lam, t_max=100, variant=variant)
        gb, gi, gps = gpu_decode(code, y, sig, gp, seed=4)
        ob, _, _ = O.decode_f32(code, y, sig, op, seed=4, threads=THREADS)
        eps[name] = dg.convergence_error(code, y, gb, cw, y_max=2.5)
        assert eps[name] == dg.convergence_error(code, y, ob, cw, y_max=2.5)
        f = dg.objective(code, y, gb, y_max=2.5)
        assert np.allclose(f[gps == 1], dg.f_max(code, y, gb, y_max=2.5)[gps == 1])
    assert eps["M-NGDBF"] > eps["M-GDBF"] and eps["AT-NGDBF"] > eps["M-GDBF"]
    assert eps["M-NGDBF uniform"] > eps["M-GDBF"]


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 3 | U])
def test_plain_per_iteration_form(O, variant):
    """The plain per-iteration kernels give ngdbf_decode's results bit for bit (and the reference
    decoder's), on a small code, the (3,6) N=1008 code and the (6,32) N=2048 code."""
    for code, F, eb, kw in ((wl.peg_code(96, 48, 3, seed=11), 150, 2.5, dict(lam=0.95, t_max=60, smooth_window=16)),
                            (wl.code_c1(), 300, 3.5, dict(lam=0.99, t_max=100, smooth_window=40)),
                            (wl.code_c2(), 120, 3.75, dict(w=0.1875, theta=-0.7, eta=0.65, lam=0.993, y_max=2.0,
                                                           t_max=200, smooth_window=64))):
        y, _, sig = wl.frames(code, F, eb, seed=48)
        gp, op = params_pair(variant=variant, **kw)
        dc = ngdbf.DeviceCode.from_code(code)
        try:
            yt = torch.from_numpy(y).cuda()
            a = [t.cpu().numpy() for t in dc.decode_plain(yt, sig, gp, seed=5, frame_offset=9)]
            assert ngdbf.ngdbf_last_launch()["kernels"] == 3 * gp.t_max + 3
            b = [t.cpu().numpy() for t in dc.decode(yt, sig, gp, seed=5, frame_offset=9)]
        finally:
            dc.close()
        for u, v, name in zip(a, b, ("bits", "iters", "pass")):
            assert np.array_equal(u, v), f"{code.name}: {name} differ from ngdbf_decode"
        ob, oi, ops = O.decode_f32(code, y[:40], sig, op, seed=5, frame_offset=9, threads=THREADS)
        assert np.array_equal(a[0][:40], ob) and np.array_equal(a[1][:40], oi) and np.array_equal(a[2][:40], ops)


def test_plain_form_rejects_what_it_lacks():
    code = wl.peg_code(96, 48, 3, seed=11)
    dc = ngdbf.DeviceCode.from_code(code)
    try:
        y = torch.zeros((4, 96), dtype=torch.float32, device="cuda")
        for kw in (dict(variant=4), dict(precision=ngdbf.NGDBF_FP16)):
            with pytest.raises(ngdbf.NgdbfError) as e:
                dc.decode_plain(y, 0.5, ngdbf.make_params(**kw))
            assert e.value.status == ngdbf.NGDBF_ERR_UNSUPPORTED
    finally:
        dc.close()
