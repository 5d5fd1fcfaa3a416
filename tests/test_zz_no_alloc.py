"""ngdbf_decode_noalloc: the decode for callers that cannot allocate device memory.

Some callers may not allocate while they run -- a receiver with a fixed memory
plan that forbids cudaMalloc after start-up (it can synchronize the device and
its latency is unbounded), or an application whose own allocator owns the
device memory.  ngdbf_decode_noalloc serves them with a static device array
instead of pool memory.  This test calls it twice in a row through the C ABI
and checks each result bit-for-bit against ngdbf_decode, the tolerance every
parity test here uses.  The second call uses a longer code whose per-slot
state lives in the static array too, so the array is reused with another
layout and a launch that is cut down to fit it.  It also checks the property
the entry point exists for: across a call, neither the library's scratch pool
(its high-water mark, reset before the call) nor the device's free memory
nor torch's allocator moves, while the same check sees ngdbf_decode's pool
allocation.
"""
import numpy as np
import pytest

from paper_1402_2773_gb300 import ngdbf, workload as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_2773_gb300 import _build
    _build.build_cuda()
    ngdbf.load()
    torch.cuda.set_device(0)


def _run(entry, code_handle, y, sigma, params, seed, offset, n):
    F = y.shape[0]
    bits = torch.empty((F, (n + 7) // 8), dtype=torch.uint8, device="cuda")
    iters = torch.empty(F, dtype=torch.int32, device="cuda")
    pas = torch.empty(F, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    entry(code_handle, y.data_ptr(), F, float(sigma), params, seed, offset,
          bits.data_ptr(), iters.data_ptr(), pas.data_ptr(), stream)
    torch.cuda.synchronize()
    return bits.cpu().numpy(), iters.cpu().numpy(), pas.cpu().numpy(), ngdbf.ngdbf_last_launch()


def test_noalloc_matches_the_allocating_entry_point_on_two_calls():
    cases = [
        # (6,32) N=2048, adaptive + smoothed: state in shared memory, full grid fits the array
        (wl.code_c2(), 3000, 4.0, ngdbf.make_params(w=0.1875, theta=-0.7, eta=0.65, lam=0.993, y_max=2.0,
                                                    t_max=300, smooth_window=64, variant=3)),
        # (3,15) N=8192, adaptive + smoothed: state in the static array, grid cut to fit it
        (wl.peg_code(8192, 1639, 3, seed=1), 1200, 3.5, ngdbf.make_params(lam=0.99, t_max=150,
                                                                         smooth_window=40, variant=3)),
    ]
    for call, (code, F, ebn0, params) in enumerate(cases):
        y_np, _, sigma = wl.frames(code, F, ebn0, seed=40 + call)
        y = torch.from_numpy(y_np).cuda()
        dc = ngdbf.DeviceCode.from_code(code)
        try:
            got = _run(ngdbf.ngdbf_decode_noalloc, dc.handle, y, sigma, params, 9, 100 * call, code.n)
            ref = _run(ngdbf.ngdbf_decode, dc.handle, y, sigma, params, 9, 100 * call, code.n)
        finally:
            dc.close()
        # a repeated no-alloc call takes nothing from the pool, the device or torch's allocator
        bits, iters, pas = (torch.empty((F, (code.n + 7) // 8), dtype=torch.uint8, device="cuda"),
                            torch.empty(F, dtype=torch.int32, device="cuda"),
                            torch.empty(F, dtype=torch.uint8, device="cuda"))
        dc = ngdbf.DeviceCode.from_code(code)
        try:
            stream = torch.cuda.current_stream().cuda_stream
            args = (dc.handle, y.data_ptr(), F, float(sigma), params, 9, 100 * call, bits.data_ptr(),
                    iters.data_ptr(), pas.data_ptr(), stream)
            torch.cuda.synchronize()
            now0, _ = ngdbf.ngdbf_pool_usage(reset_high=True)
            free0, torch0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
            ngdbf.ngdbf_decode_noalloc(*args)
            torch.cuda.synchronize()
            now1, high1 = ngdbf.ngdbf_pool_usage()
            assert (now1, high1) == (now0, now0), "ngdbf_decode_noalloc took scratch from the pool"
            assert torch.cuda.mem_get_info()[0] == free0 and torch.cuda.memory_allocated() == torch0
            ngdbf.ngdbf_pool_usage(reset_high=True)
            ngdbf.ngdbf_decode(*args)                       # control: the pool path is visible
            torch.cuda.synchronize()
            assert ngdbf.ngdbf_pool_usage()[1] > now0
        finally:
            dc.close()
        for a, b, name in zip(got[:3], ref[:3], ("bits", "iters", "pass")):
            assert np.array_equal(a, b), f"call {call}: {name} differ from ngdbf_decode"
        launch = got[3]
        per_cta = code.n * 32 * 4 + (0 if launch["state_in_smem"] else code.n * 32 * 2)
        assert launch["grid"] * per_cta <= ngdbf.NGDBF_NOALLOC_SCRATCH_BYTES
        if call == 1:
            assert launch["state_in_smem"] == 0 and launch["grid"] < ref[3]["grid"]
