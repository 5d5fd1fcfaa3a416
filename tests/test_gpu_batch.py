"""Job tables: several codes in one persistent launch, bit-exact against the reference decoder
and against one ngdbf_decode per job."""
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


def wide_code():
    rng = np.random.default_rng(5)
    n, m = 203, 101
    H = np.zeros((m, n), np.uint8)
    for k in range(n):
        H[rng.choice(m, size=int(rng.integers(2, 6)), replace=False), k] = 1
    H[:9, 0] = 1
    for i in np.nonzero(H.sum(1) == 0)[0]:
        H[i, rng.integers(n)] = 1
    return wl.code_from_dense(H)


def make_jobs(specs, variant, precision=ngdbf.NGDBF_FP32, q_bits=0):
    """specs: (code, frames, ebn0, t_max, theta, lam, w, eta, data seed, frame offset)."""
    jobs = []
    for code, F, eb, T, theta, lam, w, eta, dseed, off in specs:
        y, _, sig = wl.frames(code, F, eb, seed=dseed)
        kw = dict(w=w, theta=theta, eta=eta, lam=lam, y_max=2.5, t_max=T, smooth_window=min(64, T),
                  variant=variant, precision=precision, q_bits=q_bits)
        jobs.append(dict(code=code, y=y, sigma=sig, gp=ngdbf.make_params(**kw), op=oracle.make_params(**kw),
                         off=off))
    return jobs


def run_batch(jobs, seed, flags):
    dcs = [ngdbf.DeviceCode.from_code(j["code"]) for j in jobs]
    ys = [torch.from_numpy(j["y"]).cuda() for j in jobs]
    b = ngdbf.Batch([(dc, y, j["sigma"], j["gp"], j["off"]) for dc, y, j in zip(dcs, ys, jobs)],
                    seed=seed, flags=flags)
    outs = b.launch()
    torch.cuda.synchronize()
    res = [tuple(t.cpu().numpy() for t in o) for o in outs]
    info = ngdbf.ngdbf_last_launch()
    outs2 = b.launch()                      # a second launch gives the same results
    torch.cuda.synchronize()
    res2 = [tuple(t.cpu().numpy() for t in o) for o in outs2]
    for r, r2 in zip(res, res2):
        assert all((a == c).all() for a, c in zip(r, r2))
    single = []
    for dc, y, j in zip(dcs, ys, jobs):
        single.append(tuple(t.cpu().numpy() for t in dc.decode(y, j["sigma"], j["gp"], seed=seed,
                                                              frame_offset=j["off"])))
    torch.cuda.synchronize()
    b.close()
    for dc in dcs:
        dc.close()
    return res, single, info


def check(O, jobs, seed, flags=ngdbf.NGDBF_BATCH_GRAPH):
    res, single, info = run_batch(jobs, seed, flags)
    for j, r, s in zip(jobs, res, single):
        assert all((a == c).all() for a, c in zip(r, s)), "batch result differs from ngdbf_decode"
        if j["y"].shape[0]:
            ob, oi, op = O.decode_f32(j["code"], j["y"], j["sigma"], j["op"], seed=seed, frame_offset=j["off"],
                                      threads=THREADS)
            assert (r[0] == ob).all() and (r[1] == oi).all() and (r[2] == op).all(), "batch differs from oracle"
    return info


def mix(scale=1):
    return [
        (wl.peg_code(504, 252, 3, seed=1), 300 * scale, 3.0, 100, -0.9, 0.99, 0.75, 0.96, 1, 0),
        (wl.code_c1(), 257 * scale, 3.5, 160, -0.8, 0.98, 0.7, 0.9, 2, 1000),
        (wl.peg_code(1024, 512, 4, seed=1), 130 * scale, 2.8, 200, -0.9, 0.99, 0.75, 0.8, 3, 5),
        (wl.code_c2(), 90 * scale, 4.0, 300, -0.7, 0.993, 0.1875, 0.65, 4, 77),
        (wide_code(), 61 * scale, 3.0, 120, -0.6, 0.97, 0.6, 0.9, 5, 0),
    ]


@pytest.mark.parametrize("variant", [0, 3])
def test_mixed_codes_one_launch(O, variant):
    info = check(O, make_jobs(mix(), variant), seed=9)
    assert info["kernels"] == 1


def test_tuned_and_direct_launch(O):
    check(O, make_jobs(mix(), 1), seed=3, flags=ngdbf.NGDBF_BATCH_TUNE)
    check(O, make_jobs(mix(), 2), seed=4, flags=0)


@pytest.mark.parametrize("prec", [dict(precision=ngdbf.NGDBF_FP16), dict(precision=ngdbf.NGDBF_FIX, q_bits=8)],
                         ids=["fp16", "fix8"])
def test_mixed_codes_reduced_precision(O, prec):
    check(O, make_jobs(mix(), 3, **prec), seed=5)


def test_state_in_global_memory_for_the_whole_table(O):
    specs = mix()[:2] + [(wl.peg_code(8192, 1639, 3, seed=1), 40, 3.0, 80, -0.9, 0.99, 0.75, 0.9, 6, 9)]
    info = check(O, make_jobs(specs, 3), seed=7)
    assert info["state_in_smem"] == 0


def test_many_small_jobs_and_empty_jobs(O):
    code = wl.peg_code(504, 252, 3, seed=1)
    specs = [(code, int(f), 3.2, 60, -0.9, 0.98, 0.75, 0.9, 100 + i, 50 * i)
             for i, f in enumerate([0, 1, 5, 33, 0, 2] + [3] * 200)]
    check(O, make_jobs(specs, 3), seed=8)


def test_mixed_variants_are_rejected():
    code = wl.peg_code(504, 252, 3, seed=1)
    dc = ngdbf.DeviceCode.from_code(code)
    y = torch.zeros((4, code.n), dtype=torch.float32, device="cuda")
    with pytest.raises(ngdbf.NgdbfError) as e:
        ngdbf.Batch([(dc, y, 0.5, ngdbf.make_params(variant=0), 0), (dc, y, 0.5, ngdbf.make_params(variant=1), 0)])
    assert e.value.status == ngdbf.NGDBF_ERR_UNSUPPORTED
    dc.close()


def _table_every_shape(O, specs, variant, precision=ngdbf.NGDBF_FP32, q_bits=0, seed=3, min_cluster=2):
    """Decodes the table under every candidate launch shape; each result must equal one
    ngdbf_decode per job bit for bit (and, for a sample of frames, the reference decoder)."""
    jobs = make_jobs(specs, variant, precision, q_bits)
    dcs = [ngdbf.DeviceCode.from_code(j["code"]) for j in jobs]
    ys = [torch.from_numpy(j["y"]).cuda() for j in jobs]
    try:
        b = ngdbf.Batch([(dc, y, j["sigma"], j["gp"], j["off"]) for dc, y, j in zip(dcs, ys, jobs)],
                        seed=seed, flags=ngdbf.NGDBF_BATCH_GRAPH)
        single = [tuple(t.cpu().numpy() for t in dc.decode(y, j["sigma"], j["gp"], seed=seed,
                                                          frame_offset=j["off"]))
                  for dc, y, j in zip(dcs, ys, jobs)]
        shapes = b.shapes()
        clusters = sorted({sh["cluster"] for sh in shapes})
        assert max(clusters) >= min_cluster, shapes
        for k, sh in enumerate(shapes):
            b.use_shape(k)
            outs = b.launch()
            torch.cuda.synchronize()
            for jn, (o, ref) in enumerate(zip(outs, single)):
                got = tuple(t.cpu().numpy() for t in o)
                for a, c, name in zip(got, ref, ("bits", "iters", "pass")):
                    assert np.array_equal(a, c), f"shape {sh}, job {jn}: {name} differ"
            assert b.shape()["cluster"] == sh["cluster"]
        b.close()
    finally:
        for dc in dcs:
            dc.close()
    # the per-job decodes themselves against the reference decoder on a few frames
    for j, ref in zip(jobs, single):
        F = min(24, j["y"].shape[0])
        ob, oi, ops = O.decode_f32(j["code"], j["y"][:F], j["sigma"], j["op"], seed=seed, frame_offset=j["off"],
                                   threads=THREADS)
        assert np.array_equal(ob, ref[0][:F]) and np.array_equal(oi, ref[1][:F]) and np.array_equal(ops, ref[2][:F])
    return clusters


def _cluster_specs():
    return [(wl.peg_code(504, 252, 3, seed=1), 70, 3.0, 120, -0.9, 0.99, 0.75, 0.95, 61, 0),
            (wl.peg_code(2048, 384, 6, seed=1), 90, 3.75, 150, -0.7, 0.993, 0.1875, 0.65, 62, 10 ** 6),
            (wl.peg_code(4096, 2048, 4, seed=1), 40, 2.5, 100, -0.9, 0.98, 0.75, 0.7, 63, 5),
            (wl.peg_code(8192, 1639, 3, seed=1), 50, 3.0, 120, -0.7, 0.99, 0.5, 0.8, 64, 77)]


@pytest.mark.parametrize("variant", [3, 0, 2, 6, 4, 3 | ngdbf.NGDBF_UNIFORM])
def test_cluster_split_every_shape(O, variant):
    """Codes of 2048 symbols or more split over thread-block clusters of 2, 4 and 8 CTAs (the
    decision words exchanged through distributed shared memory), smaller ones decoded CTA by CTA,
    every placement and block size: identical to one ngdbf_decode per job."""
    clusters = _table_every_shape(O, _cluster_specs(), variant)
    assert clusters[0] == 1


@pytest.mark.parametrize("precision,q_bits", [(ngdbf.NGDBF_FP16, 0), (ngdbf.NGDBF_FIXACC, 8)])
def test_cluster_split_precisions(O, precision, q_bits):
    _table_every_shape(O, _cluster_specs()[1:3], 3, precision, q_bits)


def test_cluster_split_ragged_code():
    """A split code whose length is not a multiple of 32 (the last CTA's range ends mid-group)."""
    H = wl.peg_code(2600, 1300, 3, seed=2).dense()[:, :2598]
    H = H[H.sum(axis=1) > 0]
    code = wl.code_from_dense(H)
    O = oracle.load()
    _table_every_shape(O, [(code, 75, 2.5, 90, -0.9, 0.99, 0.75, 0.95, 65, 3),
                           (wl.peg_code(96, 48, 3, seed=11), 40, 2.5, 60, -0.9, 0.99, 0.75, 0.95, 66, 0)], 3)
