"""Serving loop: requests of different codes and sizes admitted under a memory budget into a
resident persistent kernel (continuous batching); every result equals the request decoded alone."""
import os
import threading

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
def codes():
    return [wl.peg_code(504, 252, 3, seed=1), wl.code_c1(), wl.peg_code(1024, 512, 4, seed=1), wl.code_c2()]


def requests(codes, count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for r in range(count):
        c = int(rng.integers(len(codes)))
        code = codes[c]
        F = int(rng.integers(1, 300))
        eb = float(rng.uniform(3.0, 4.5))
        T = int(rng.integers(60, 200))
        y, _, sig = wl.frames(code, F, eb, seed=1000 + r)
        kw = dict(w=0.75 if c < 3 else 0.1875, theta=-0.9 if c < 3 else -0.7, eta=0.9 if c < 3 else 0.65,
                  lam=0.99, y_max=2.5 if c < 3 else 2.0, t_max=T, smooth_window=64, variant=3)
        out.append(dict(c=c, y=torch.from_numpy(y).pin_memory(), sigma=sig, kw=kw, off=10_000 * r))
    return out


def decode_alone(dcs, reqs, seed):
    res = []
    for q in reqs:
        dc = dcs[q["c"]]
        b, i, p = dc.decode(q["y"].cuda(), q["sigma"], ngdbf.make_params(**q["kw"]), seed=seed, frame_offset=q["off"])
        torch.cuda.synchronize()
        res.append((b.cpu().numpy(), i.cpu().numpy(), p.cpu().numpy()))
    return res


def serve(dcs, reqs, budget, inflight, max_jobs, seed, threads=1):
    srv = ngdbf.Server(budget, max_inflight=inflight, max_jobs=max_jobs, seed=seed)
    outs = [None] * len(reqs)

    def submit(idx):
        for k in idx:
            q = reqs[k]
            F = q["y"].shape[0]
            n = dcs[q["c"]].n
            buf = (torch.empty((F, (n + 7) // 8), dtype=torch.uint8).pin_memory(),
                   torch.empty(F, dtype=torch.int32).pin_memory(), torch.empty(F, dtype=torch.uint8).pin_memory())
            _, outs[k] = srv.submit(dcs[q["c"]], q["y"], q["sigma"], ngdbf.make_params(**q["kw"]), q["off"], out=buf)

    parts = [list(range(t, len(reqs), threads)) for t in range(threads)]
    ths = [threading.Thread(target=submit, args=(p,)) for p in parts]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    srv.wait(600)
    done = srv.poll()
    stats = srv.stats()
    srv.close()
    return [tuple(o.numpy() for o in out) for out in outs], done, stats


def test_mix_equals_alone(codes):
    dcs = [ngdbf.DeviceCode.from_code(c) for c in codes]
    reqs = requests(codes, 60, seed=1)
    alone = decode_alone(dcs, reqs, seed=5)
    got, done, stats = serve(dcs, reqs, budget=2 << 30, inflight=4, max_jobs=16, seed=5, threads=3)
    assert len(done) == len(reqs) and all(st == 0 for _, _, st in done)
    for g, a in zip(got, alone):
        assert all((x == y).all() for x, y in zip(g, a)), "served result differs from the request alone"
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    assert stats["launches"] >= 1 and stats["peak_requests_on_device"] >= 2
    assert stats["peak_bytes_in_use"] <= 2 << 30
    # a few requests against the reference decoder
    O = oracle.load()
    for q, g in list(zip(reqs, got))[:6]:
        ob, oi, op = O.decode_f32(codes[q["c"]], q["y"].numpy(), q["sigma"], oracle.make_params(**q["kw"]), seed=5,
                                  frame_offset=q["off"], threads=THREADS)
        assert (g[0] == ob).all() and (g[1] == oi).all() and (g[2] == op).all()
    for dc in dcs:
        dc.close()


def test_tight_budget_and_oversized_request(codes):
    dcs = [ngdbf.DeviceCode.from_code(c) for c in codes]
    reqs = requests(codes, 12, seed=2)
    alone = decode_alone(dcs, reqs, seed=6)
    budget = 160 << 20                     # about one launch at a time
    big = dict(c=3, y=torch.zeros((20000, codes[3].n), dtype=torch.float32).pin_memory(), sigma=0.5,
               kw=reqs[0]["kw"] | dict(w=0.1875), off=0)
    got, done, stats = serve(dcs, reqs + [big], budget=budget, inflight=3, max_jobs=4, seed=6)
    status = {rid: st for rid, _, st in done}
    assert len(done) == len(reqs) + 1
    assert sorted(status.values()).count(ngdbf.NGDBF_ERR_OOM) == 1      # the oversized request only
    for g, a in zip(got[:-1], alone):
        assert all((x == y).all() for x, y in zip(g, a))
    assert stats["peak_bytes_in_use"] <= budget and stats["failed"] == 1
    for dc in dcs:
        dc.close()


def test_requests_join_a_running_launch(codes):
    """A long request keeps the resident kernel busy; requests submitted while it runs are
    published into that same launch (no second launch), their work overlaps it on the device,
    and every result equals the request decoded alone."""
    import time
    dcs = [ngdbf.DeviceCode.from_code(c) for c in codes]
    kw = dict(w=0.1875, theta=-0.7, eta=0.65, lam=0.993, y_max=2.0, t_max=300, smooth_window=64, variant=3)
    y_big, _, sig_big = wl.frames(codes[3], 60000, 3.5, seed=77)
    big = dict(c=3, y=torch.from_numpy(y_big).pin_memory(), sigma=sig_big, kw=kw, off=7)
    small = []
    for k in range(12):
        y, _, sig = wl.frames(codes[3], 50 + 10 * k, 4.0, seed=90 + k)
        small.append(dict(c=3, y=torch.from_numpy(y).pin_memory(), sigma=sig, kw=kw, off=10 ** 6 * (k + 1)))
    alone = decode_alone(dcs, [big] + small, seed=8)
    srv = ngdbf.Server(8 << 30, max_inflight=2, max_jobs=64, seed=8)
    outs = []
    for q in [big] + small:
        F, n = q["y"].shape[0], codes[3].n
        outs.append((torch.empty((F, (n + 7) // 8), dtype=torch.uint8).pin_memory(),
                     torch.empty(F, dtype=torch.int32).pin_memory(), torch.empty(F, dtype=torch.uint8).pin_memory()))
    ids = [srv.submit(dcs[3], big["y"], big["sigma"], ngdbf.make_params(**big["kw"]), big["off"], out=outs[0])[0]]
    t0 = time.time()
    while srv.stats()["launches"] == 0 and time.time() - t0 < 30:   # the big request is on the device
        time.sleep(0.0005)
    for q, o in zip(small, outs[1:]):
        ids.append(srv.submit(dcs[3], q["y"], q["sigma"], ngdbf.make_params(**q["kw"]), q["off"], out=o)[0])
    srv.wait(600)
    done = {rid: st for rid, _, st in srv.poll()}
    stats = srv.stats()
    srv.close()
    assert all(done[i] == 0 for i in ids)
    for o, a in zip(outs, alone):
        assert all((x.numpy() == y).all() for x, y in zip(o, a)), "served result differs from the request alone"
    assert stats["launches"] == 1, stats
    assert stats["admitted_into_running"] >= len(small), stats
    assert stats["peak_requests_on_device"] >= 2, stats
    for dc in dcs:
        dc.close()


def test_chained_requests_of_one_code(codes):
    """Many requests of the same code and parameters pending at once (different samples, sigma,
    sizes and frame offsets): CTAs decode frames of several of them in their slots at once, and
    every result still equals the request decoded alone (per-slot sigma, offset, outputs and
    completion counts).  A second parameter set in the mix keeps its own chain."""
    dcs = [ngdbf.DeviceCode.from_code(c) for c in codes]
    rng = np.random.default_rng(21)
    kw_a = dict(w=0.1875, theta=-0.7, eta=0.65, lam=0.993, y_max=2.0, t_max=150, smooth_window=64, variant=3)
    kw_b = dict(w=0.75, theta=-0.9, eta=0.9, lam=0.99, y_max=2.5, t_max=120, smooth_window=64, variant=3)
    reqs = []
    for r in range(96):
        c, kw = (3, kw_a) if r % 4 else (1, kw_b)
        F = int(rng.integers(1, 120))
        y, _, sig = wl.frames(codes[c], F, float(rng.uniform(3.0, 4.5)), seed=3000 + r)
        reqs.append(dict(c=c, y=torch.from_numpy(y).pin_memory(), sigma=sig, kw=kw, off=1000 * r + 17))
    alone = decode_alone(dcs, reqs, seed=12)
    got, done, stats = serve(dcs, reqs, budget=4 << 30, inflight=4, max_jobs=256, seed=12)
    assert len(done) == len(reqs) and all(st == 0 for _, _, st in done)
    for g, a in zip(got, alone):
        assert all((x == y).all() for x, y in zip(g, a)), "served result differs from the request alone"
    assert stats["peak_requests_on_device"] >= 16, stats
    for dc in dcs:
        dc.close()


def test_direct_copy_mode_serves_the_same_results(codes):
    """The server with direct copies (no staging) gives the same results as each request alone."""
    dcs = [ngdbf.DeviceCode.from_code(c) for c in codes]
    reqs = requests(codes, 16, seed=7)
    alone = decode_alone(dcs, reqs, seed=9)
    old = ngdbf.ngdbf_get_host_copy_mode()
    try:
        ngdbf.ngdbf_set_host_copy_mode(ngdbf.NGDBF_HOST_COPY_DIRECT)
        got, done, stats = serve(dcs, reqs, budget=1 << 30, inflight=2, max_jobs=8, seed=9)
    finally:
        ngdbf.ngdbf_set_host_copy_mode(old)
    assert len(done) == len(reqs) and all(st == 0 for _, _, st in done)
    for g, a in zip(got, alone):
        assert all((x == y).all() for x, y in zip(g, a))
    for dc in dcs:
        dc.close()


def test_requests_across_kernel_retirements(codes):
    """Requests arriving with gaps longer than the idle time: the resident kernel retires as a
    whole between them and is launched again; a request that arrives while it retires waits for
    the next launch.  Every result equals the request decoded alone."""
    import time
    dcs = [ngdbf.DeviceCode.from_code(c) for c in codes]
    reqs = requests(codes, 10, seed=11)
    alone = decode_alone(dcs, reqs, seed=13)
    srv = ngdbf.Server(1 << 30, max_inflight=2, max_jobs=16, seed=13)
    outs = []
    for k, q in enumerate(reqs):
        F, n = q["y"].shape[0], dcs[q["c"]].n
        buf = (torch.empty((F, (n + 7) // 8), dtype=torch.uint8).pin_memory(),
               torch.empty(F, dtype=torch.int32).pin_memory(), torch.empty(F, dtype=torch.uint8).pin_memory())
        srv.submit(dcs[q["c"]], q["y"], q["sigma"], ngdbf.make_params(**q["kw"]), q["off"], out=buf)
        outs.append(buf)
        time.sleep(0.005 if k % 3 == 2 else 0.045)     # mostly longer than the idle time
    srv.wait(600)
    done = srv.poll()
    stats = srv.stats()
    srv.close()
    assert len(done) == len(reqs) and all(st == 0 for _, _, st in done)
    for o, a in zip(outs, alone):
        assert all((x.numpy() == y).all() for x, y in zip(o, a))
    assert stats["launches"] >= 3, stats
    for dc in dcs:
        dc.close()


@pytest.mark.parametrize("prec", [dict(), dict(precision=ngdbf.NGDBF_FP16), dict(precision=ngdbf.NGDBF_FIX, q_bits=8),
                                  dict(precision=ngdbf.NGDBF_FIXACC, q_bits=8)], ids=["fp32", "fp16", "fix8", "fixacc8"])
def test_mix_with_a_code_whose_state_is_off_chip(codes, prec):
    """A mix whose largest code (N = 8192) keeps its slot state in global memory: the resident
    kernel decodes every request in a layout of its own code, so the smaller codes' requests keep
    their state in shared memory in the same launch; every result equals the request decoded
    alone, and a few equal the reference decoder (in every held precision)."""
    big_code = wl.peg_code(8192, 1639, 3, seed=1)
    mix = [codes[0], codes[3], big_code]
    dcs = [ngdbf.DeviceCode.from_code(c) for c in mix]
    kws = [dict(w=0.75, theta=-0.9, eta=0.9, lam=0.99, y_max=2.5),
           dict(w=0.1875, theta=-0.7, eta=0.65, lam=0.993, y_max=2.0),
           dict(w=0.5, theta=-0.7, eta=0.8, lam=0.99, y_max=2.5)]
    rng = np.random.default_rng(31)
    reqs = []
    for r in range(30):
        c = 2 if r % 5 == 0 else int(rng.integers(2))      # the large code first, then every fifth
        F = int(rng.integers(1, 200 if c < 2 else 48))
        y, _, sig = wl.frames(mix[c], F, float(rng.uniform(3.5, 4.5)), seed=4000 + r)
        kw = kws[c] | dict(t_max=int(rng.integers(60, 200)), smooth_window=64, variant=3) | prec
        reqs.append(dict(c=c, y=torch.from_numpy(y).pin_memory(), sigma=sig, kw=kw, off=5000 * r + 3))
    alone = decode_alone(dcs, reqs[:1], seed=14)
    assert ngdbf.ngdbf_last_launch()["state_in_smem"] == 0      # the large code's state is off chip
    alone += decode_alone(dcs, reqs[1:], seed=14)
    got, done, stats = serve(dcs, reqs, budget=4 << 30, inflight=4, max_jobs=64, seed=14)
    assert len(done) == len(reqs) and all(st == 0 for _, _, st in done)
    for g, a in zip(got, alone):
        assert all((x == y).all() for x, y in zip(g, a)), "served result differs from the request alone"
    O = oracle.load()
    for q, g in [(q, g) for q, g in zip(reqs, got) if q["c"] < 2][:4]:
        ob, oi, op = O.decode_f32(mix[q["c"]], q["y"].numpy(), q["sigma"], oracle.make_params(**q["kw"]), seed=14,
                                  frame_offset=q["off"], threads=THREADS)
        assert (g[0] == ob).all() and (g[1] == oi).all() and (g[2] == op).all()
    for dc in dcs:
        dc.close()
