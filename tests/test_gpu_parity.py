"""CUDA decoder vs the FP32 reference decoder: bit-exact bits, iteration counts and pass flags.

All calls go through the C ABI (libngdbf.so via ctypes).  Cases span several
32-slot CTAs, ragged frame counts and code lengths, irregular degrees, every
variant, both placements of the per-slot state (shared or global memory),
the edge values of every parameter, and the full-size workloads on sampled
frames.
"""
import ctypes
import os

import numpy as np
import pytest

import oracle
from paper_1402_2773_gb300 import ngdbf, workload as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1


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
    assert bad.size == 0, (f"{bad.size}/{y.shape[0]} frames differ, first {bad[:5]}: "
                           f"gpu iters {gi[bad[:5]]} oracle {oi[bad[:5]]}")
    return oi, ops


def irregular_code(n, m, seed):
    """Random H with symbol degrees 2..5 and every check used (degrees ragged on both sides)."""
    rng = np.random.default_rng(seed)
    H = np.zeros((m, n), np.uint8)
    for k in range(n):
        H[rng.choice(m, size=int(rng.integers(2, 6)), replace=False), k] = 1
    for i in np.nonzero(H.sum(1) == 0)[0]:
        H[i, rng.integers(n)] = 1
    return wl.code_from_dense(H, name=f"irregular_{n}x{m}")


HAMMING = np.array([[1, 1, 0, 1, 1, 0, 0], [1, 0, 1, 1, 0, 1, 0], [0, 1, 1, 1, 0, 0, 1]], np.uint8)


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_hamming_ragged(O, variant):
    code = wl.code_from_dense(HAMMING)
    y, _, sig = wl.frames(code, 45, 1.0, seed=3)
    assert_parity(O, code, y, sig, seed=2, variant=variant, lam=0.9, t_max=20, smooth_window=7)


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_small_peg_code(O, variant):
    code = wl.peg_code(96, 48, 3, seed=11)
    y, _, sig = wl.frames(code, 100, 2.5, seed=4)
    assert_parity(O, code, y, sig, seed=9, variant=variant, lam=0.95, t_max=60, smooth_window=16)


@pytest.mark.parametrize("variant", [0, 3])
def test_irregular_code(O, variant):
    code = irregular_code(203, 101, seed=5)
    y, _, sig = wl.frames(code, 70, 3.0, seed=6)
    assert_parity(O, code, y, sig, seed=3, variant=variant, lam=0.97, t_max=40, smooth_window=9)


def test_c1_plain_full(O):
    """(3,6) N=1008, 10^4 frames at 4.0 dB, plain M-NGDBF: every frame compared."""
    code = wl.code_c1()
    y, cw, sig = wl.frames(code, 10000, 4.0, seed=1)
    it, ps = assert_parity(O, code, y, sig, seed=1, w=0.75, theta=-0.9, eta=0.96, t_max=100)
    assert 10 < it.mean() < 80 and 0.5 < ps.mean() < 1.0


@pytest.mark.parametrize("ebn0", [3.5, 4.0, 4.5])
def test_c2_smoothed_adaptive(O, ebn0):
    """(6,32) N=2048 SM-NGDBF with adaptation, T=300, W=64 (shared-memory state)."""
    code = wl.code_c2()
    y, _, sig = wl.frames(code, 300, ebn0, seed=2)
    assert_parity(O, code, y, sig, seed=7, w=0.1875, theta=-0.7, eta=0.65, lam=0.993, y_max=2.0,
                  t_max=300, smooth_window=64, variant=3)
    assert ngdbf.ngdbf_last_launch()["state_in_smem"] == 1


def test_global_state_path(O):
    """(3,15) N=8192 and (4,8) N=4096: per-slot state too large for shared memory."""
    code = wl.peg_code(8192, 1639, 3, seed=1)
    y, _, sig = wl.frames(code, 40, 3.0, seed=8)
    assert_parity(O, code, y, sig, seed=4, lam=0.99, t_max=120, smooth_window=32, variant=3)
    assert ngdbf.ngdbf_last_launch()["state_in_smem"] == 0
    code = wl.peg_code(4096, 2048, 4, seed=1)
    y, _, sig = wl.frames(code, 40, 2.5, seed=8)
    assert_parity(O, code, y, sig, seed=4, lam=0.98, t_max=100, smooth_window=20, variant=1)
    assert ngdbf.ngdbf_last_launch()["state_in_smem"] == 0


@pytest.mark.parametrize("n", [2250, 2400])
def test_tables_in_global_memory(O, n):
    """The per-slot state fits shared memory only with one adjacency table (N=2250) or both
    (N=2400) in global memory."""
    code = wl.peg_code(n, n // 2, 3, seed=2)
    y, _, sig = wl.frames(code, 40, 2.5, seed=1)
    assert_parity(O, code, y, sig, seed=4, lam=0.98, t_max=60, variant=1)
    info = ngdbf.ngdbf_last_launch()
    assert info["state_in_smem"] == 1 and info["tables_in_smem"] in ((1, 2) if n == 2250 else (0,))


@pytest.mark.parametrize("kw", [
    dict(t_max=0), dict(t_max=1), dict(t_max=511, smooth_window=126, variant=3, lam=0.999),
    dict(eta=0.0), dict(eta=0.0, variant=1, lam=0.9), dict(y_max=0.0), dict(y_max=float("inf")),
    dict(smooth_window=200 // 2, t_max=30, variant=2), dict(smooth_window=0, variant=2, t_max=50),
    dict(theta=0.5), dict(w=3.0), dict(lam=1.0, variant=1),
], ids=lambda d: ",".join(f"{k}={v}" for k, v in d.items()))
def test_parameter_edges(O, kw):
    code = wl.peg_code(504, 252, 3, seed=3)
    y, _, sig = wl.frames(code, 70, 2.8, seed=5)
    base = dict(lam=0.97, t_max=50, smooth_window=12)
    base.update(kw)
    assert_parity(O, code, y, sig, seed=6, **base)


@pytest.mark.parametrize("F", [1, 31, 32, 33, 65])
def test_ragged_frame_counts(O, F):
    code = wl.peg_code(504, 252, 3, seed=3)
    y, _, sig = wl.frames(code, F, 3.0, seed=11)
    assert_parity(O, code, y, sig, seed=1, variant=3, lam=0.97, t_max=60, smooth_window=10)


def test_zero_frames_is_a_no_op():
    code = wl.peg_code(504, 252, 3, seed=3)
    dc = ngdbf.DeviceCode.from_code(code)
    y = torch.empty((0, code.n), dtype=torch.float32, device="cuda")
    b, i, p = dc.decode(y, 0.5, ngdbf.make_params())
    torch.cuda.synchronize()
    assert b.numel() == 0 and ngdbf.ngdbf_last_launch()["kernels"] == 0
    dc.close()


def test_noiseless_frames(O):
    code = wl.code_c2()
    y, cw, _ = wl.frames(code, 64, None, seed=2)
    gp, _ = params_pair(variant=3, lam=0.99, t_max=300)
    b, i, p = gpu_decode(code, y, 0.4, gp, seed=1)
    assert (i == 0).all() and (p == 1).all() and (b == cw).all()


def test_results_independent_of_batch(O):
    """A frame decodes identically alone, at another batch position, or in a larger batch."""
    code = wl.code_c1()
    y, _, sig = wl.frames(code, 2000, 3.5, seed=13)
    gp, _ = params_pair(variant=3, lam=0.98, t_max=150)
    b, i, p = gpu_decode(code, y, sig, gp, seed=3, frame_offset=1000)
    b2, i2, p2 = gpu_decode(code, y[700:760], sig, gp, seed=3, frame_offset=1700)
    assert (b[700:760] == b2).all() and (i[700:760] == i2).all() and (p[700:760] == p2).all()
    b3, i3, p3 = gpu_decode(code, y[1234:1235], sig, gp, seed=3, frame_offset=2234)
    assert (b[1234] == b3[0]).all() and i[1234] == i3[0]


def test_passing_outputs_are_codewords():
    code = wl.code_c1()
    y, cw, sig = wl.frames(code, 4000, 3.0, seed=17)
    gp, _ = params_pair(variant=1, lam=0.98, t_max=100)
    b, i, p = gpu_decode(code, y, sig, gp, seed=3)
    H = code.dense().astype(np.int64)
    x = wl.unpack_bits(b, code.n).astype(np.int64)
    synd = (x @ H.T) % 2
    assert (synd[p == 1] == 0).all() and synd[p == 0].any(axis=1).all()


def test_host_entry_point_matches_device(O):
    code = wl.code_c1()
    y, _, sig = wl.frames(code, 1000, 3.5, seed=19)
    gp, op = params_pair(variant=3, lam=0.98, t_max=120)
    dc = ngdbf.DeviceCode.from_code(code)
    yp = torch.from_numpy(y).pin_memory()
    hb, hi, hp = dc.decode_host(yp, sig, gp, seed=5, frame_offset=3, chunk_frames=300)
    assert ngdbf.ngdbf_last_launch()["kernels"] == 4
    hb2, hi2, hp2 = dc.decode_host(y, sig, gp, seed=5, frame_offset=3)   # pageable, one chunk
    dc.close()
    ob, oi, ops = O.decode_f32(code, y, sig, op, seed=5, frame_offset=3, threads=THREADS)
    assert (hb == ob).all() and (hi == oi).all() and (hp == ops).all()
    assert (hb2 == ob).all() and (hi2 == oi).all() and (hp2 == ops).all()


PRECISIONS = [dict(precision=ngdbf.NGDBF_FP16), dict(precision=ngdbf.NGDBF_FIX, q_bits=8),
              dict(precision=ngdbf.NGDBF_FIX, q_bits=4, y_max=1.75), dict(precision=ngdbf.NGDBF_FIX, q_bits=3)]
PREC_IDS = ["fp16", "fix8", "fix4", "fix3"]


@pytest.mark.parametrize("prec", PRECISIONS, ids=PREC_IDS)
@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_precision_variants_small(O, prec, variant):
    code = wl.peg_code(504, 252, 3, seed=3)
    y, _, sig = wl.frames(code, 70, 2.8, seed=31)
    assert_parity(O, code, y, sig, seed=6, variant=variant, lam=0.97, t_max=60, smooth_window=12, **prec)


@pytest.mark.parametrize("prec", PRECISIONS[:2], ids=PREC_IDS[:2])
def test_precision_variants_workloads(O, prec):
    """(3,6) N=1008 plain at 4 dB and (6,32) N=2048 SM-NGDBF at 4 dB in FP16 and 8-bit fixed point."""
    code = wl.code_c1()
    y, _, sig = wl.frames(code, 1500, 4.0, seed=32)
    assert_parity(O, code, y, sig, seed=1, w=0.75, theta=-0.9, eta=0.96, t_max=100, **prec)
    code = wl.code_c2()
    y, _, sig = wl.frames(code, 200, 4.0, seed=33)
    assert_parity(O, code, y, sig, seed=7, w=0.1875, theta=-0.7, eta=0.65, lam=0.993, y_max=2.0,
                  t_max=300, smooth_window=64, variant=3, **prec)


@pytest.mark.parametrize("prec", PRECISIONS[:2], ids=PREC_IDS[:2])
def test_precision_variants_global_state_and_wide(O, prec):
    """State in global memory (N=8192) and symbol degree above 7 (bit-sliced counts)."""
    code = wl.peg_code(8192, 1639, 3, seed=1)
    y, _, sig = wl.frames(code, 40, 3.0, seed=34)
    assert_parity(O, code, y, sig, seed=4, lam=0.99, t_max=80, smooth_window=20, variant=3, **prec)
    code = irregular_code(203, 101, seed=5)
    H = code.dense()
    H[:, 0] = 0
    H[:9, 0] = 1                                   # one symbol of degree 9
    code = wl.code_from_dense(H)
    y, _, sig = wl.frames(code, 70, 3.0, seed=35)
    assert_parity(O, code, y, sig, seed=3, variant=3, lam=0.97, t_max=40, smooth_window=9, **prec)


@pytest.mark.parametrize("prec", [dict(), *PRECISIONS[:2]], ids=["fp32", *PREC_IDS[:2]])
@pytest.mark.parametrize("variant", [4, 6])
def test_single_bit_variant(O, variant, prec):
    """S-NGDBF (Step 3a): one flip per iteration, the least E_k (lowest k on ties)."""
    code = wl.peg_code(504, 252, 3, seed=3)
    y, _, sig = wl.frames(code, 70, 4.0, seed=41)
    assert_parity(O, code, y, sig, seed=6, variant=variant, eta=1.0, t_max=100, smooth_window=20, **prec)
    code = wl.code_c1()
    y, _, sig = wl.frames(code, 100, 4.5, seed=42)
    assert_parity(O, code, y, sig, seed=6, variant=variant, eta=1.0, t_max=100, smooth_window=20, **prec)


def test_single_bit_ties_and_wide_and_global_state(O):
    # eta = 0 with dyadic samples makes equal E_k common: ties must go to the lowest k
    code = wl.peg_code(504, 252, 3, seed=3)
    rng = np.random.default_rng(43)
    y, _, _ = wl.frames(code, 64, None, seed=43)
    y = (y + rng.integers(-12, 13, size=y.shape) / 8).astype(np.float32)
    assert_parity(O, code, y, 0.5, seed=2, variant=4, eta=0.0, w=0.5, t_max=60)
    code = irregular_code(203, 101, seed=5)
    H = code.dense()
    H[:9, 0] = 1
    code = wl.code_from_dense(H)
    y, _, sig = wl.frames(code, 40, 3.5, seed=44)
    assert_parity(O, code, y, sig, seed=3, variant=6, eta=1.0, t_max=50, smooth_window=9)
    code = wl.peg_code(8192, 1639, 3, seed=1)
    y, _, sig = wl.frames(code, 8, 5.0, seed=45)
    assert_parity(O, code, y, sig, seed=3, variant=6, eta=1.0, t_max=30, smooth_window=9, w=0.5, theta=-0.7)


def test_invalid_arguments_report_status():
    code = wl.peg_code(504, 252, 3, seed=3)
    dc = ngdbf.DeviceCode.from_code(code)
    y = torch.zeros((4, code.n), dtype=torch.float32, device="cuda")
    with pytest.raises(ngdbf.NgdbfError) as e:
        dc.decode(y, 0.5, ngdbf.make_params(t_max=600))
    assert e.value.status == ngdbf.NGDBF_ERR_UNSUPPORTED
    with pytest.raises(ngdbf.NgdbfError) as e:
        dc.decode(y, 0.5, ngdbf.make_params(eta=1.5))
    assert e.value.status == ngdbf.NGDBF_ERR_INVALID_ARG
    with pytest.raises(ngdbf.NgdbfError) as e:
        dc.decode(y, -1.0, ngdbf.make_params())
    assert e.value.status == ngdbf.NGDBF_ERR_INVALID_ARG
    for bad in (dict(precision=ngdbf.NGDBF_FIX, q_bits=9), dict(precision=ngdbf.NGDBF_FIX, q_bits=8, y_max=0.0),
                dict(precision=ngdbf.NGDBF_FP16, q_bits=4), dict(precision=7), dict(variant=5), dict(variant=16)):
        with pytest.raises(ngdbf.NgdbfError) as e:
            dc.decode(y, 0.5, ngdbf.make_params(**bad))
        assert e.value.status == ngdbf.NGDBF_ERR_INVALID_ARG
    host = np.zeros((4, code.n), np.float32)
    out = torch.empty((4, 63), dtype=torch.uint8, device="cuda")
    it = torch.empty(4, dtype=torch.int32, device="cuda")
    ps = torch.empty(4, dtype=torch.uint8, device="cuda")
    with pytest.raises(ngdbf.NgdbfError) as e:      # host pointer where device memory is required
        ngdbf.ngdbf_decode(dc.handle, host.ctypes.data, 4, 0.5, ngdbf.make_params(), 1, 0,
                           out.data_ptr(), it.data_ptr(), ps.data_ptr(), 0)
    assert e.value.status == ngdbf.NGDBF_ERR_INVALID_ARG
    dc.close()


def test_code_beyond_shared_memory_is_rejected():
    """n = 12000, m = 6000: the code's tables build, but one CTA's decision, syndrome and count
    words exceed shared memory, so decoding reports UNSUPPORTED (and nothing is launched)."""
    n, m = 12000, 6000
    row_ptr = np.arange(0, 2 * m + 1, 2, dtype=np.int32)
    col_idx = np.arange(2 * m, dtype=np.int32)
    h = ctypes.c_void_p()
    i32p = ctypes.POINTER(ctypes.c_int32)
    lib = ngdbf.load()
    assert lib.ngdbf_code_create(n, m, row_ptr.ctypes.data_as(i32p), col_idx.ctypes.data_as(i32p),
                                 ctypes.byref(h)) == ngdbf.NGDBF_OK
    y = torch.zeros((4, n), dtype=torch.float32, device="cuda")
    out = torch.empty((4, (n + 7) // 8), dtype=torch.uint8, device="cuda")
    it = torch.empty(4, dtype=torch.int32, device="cuda")
    ps = torch.empty(4, dtype=torch.uint8, device="cuda")
    for variant in (0, 3):
        with pytest.raises(ngdbf.NgdbfError) as e:
            ngdbf.ngdbf_decode(h.value, y.data_ptr(), 4, 0.5, ngdbf.make_params(variant=variant), 1, 0,
                               out.data_ptr(), it.data_ptr(), ps.data_ptr(), 0)
        assert e.value.status == ngdbf.NGDBF_ERR_UNSUPPORTED and "too large" in str(e.value)
    assert lib.ngdbf_code_destroy(h) == ngdbf.NGDBF_OK


def test_full_size_c2_sampled(O):
    """10^6 frames of the (6,32) N=2048 code at 4.0 dB in the benchmark's launch shape; 1500 frames
    spread over the batch decoded by the oracle one by one (frame id = offset + index)."""
    code = wl.code_c2()
    F = 1_000_000
    y, cw, sig = wl.frames(code, F, 4.0, seed=1001, threads=THREADS)
    gp, op = params_pair(w=0.1875, theta=-0.7, eta=0.65, lam=0.993, y_max=2.0, t_max=300,
                         smooth_window=64, variant=3)
    gb, gi, gps = gpu_decode(code, y, sig, gp, seed=77, frame_offset=0)
    info = ngdbf.ngdbf_last_launch()
    assert info["grid"] == info["sm_count"] * (info["grid"] // info["sm_count"])
    idx = np.unique(np.concatenate([np.arange(0, F, F // 1000), np.arange(F - 200, F),
                                    np.nonzero(gps == 0)[0][:300]]))

    def one(f):
        ob, oi, ops = O.decode_f32(code, y[f:f + 1], sig, op, seed=77, frame_offset=int(f), threads=1)
        return f, bool((gb[f] == ob[0]).all() and gi[f] == oi[0] and gps[f] == ops[0])

    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(THREADS) as ex:
        bad = [f for f, ok in ex.map(one, idx.tolist()) if not ok]
    assert not bad, f"{len(bad)} of {idx.size} sampled frames differ, first {bad[:5]}"
    # property at full size: every passing frame is a codeword
    H = torch.from_numpy(code.dense().astype(np.float32)).cuda()
    for s in range(0, F, 100_000):
        x = torch.from_numpy(wl.unpack_bits(gb[s:s + 100_000], code.n).astype(np.float32)).cuda()
        synd = torch.remainder(x @ H.T, 2.0).amax(dim=1).cpu().numpy()
        p = gps[s:s + 100_000]
        assert (synd[p == 1] == 0).all()
