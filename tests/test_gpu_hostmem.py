"""Page-locked host blocks from ngdbf_host_alloc: pinned, usable by the host-buffer decode
(bit-identical to the same decode from torch's pinned memory), returned on free."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1402_2773_gb300 import ngdbf
from paper_1402_2773_gb300 import workload as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    return ngdbf.load()


def test_large_block_is_huge_page_aligned_and_pinned():
    hp = ngdbf.ngdbf_host_huge_page_bytes()
    nbytes = max(hp, 1 << 21) + 12345          # at least one huge page: the mapped path
    t = ngdbf.host_empty(nbytes, np.uint8)
    assert t.is_pinned()
    if hp:
        assert t.data_ptr() % hp == 0
    mapped, huge = ngdbf.ngdbf_host_block_info(t.data_ptr())
    if hp:
        assert mapped % hp == 0 and mapped >= nbytes
        assert -1 <= huge <= mapped
    t.numpy()[:] = 7
    d = t.cuda()
    assert int(d[-1].item()) == 7 and int(d.sum().item()) == 7 * nbytes


def test_small_block_and_free():
    p = ngdbf.ngdbf_host_alloc(4096)
    ngdbf.ngdbf_host_free(p)
    with pytest.raises(ngdbf.NgdbfError):
        ngdbf.ngdbf_host_free(p)                  # already returned


def test_decode_host_from_library_blocks_matches_torch_pinned():
    code = wl.code_c1()
    F = 3000
    y, _, sig = wl.frames(code, F, 3.5, seed=77)
    dc = ngdbf.DeviceCode.from_code(code)
    gp = ngdbf.make_params(w=0.75, theta=-0.9, eta=0.96, y_max=2.5, t_max=100, variant=0)
    nb = (code.n + 7) // 8
    ya = ngdbf.host_empty((F, code.n), np.float32)
    ya.numpy()[:] = y
    outs_a = (ngdbf.host_empty((F, nb), np.uint8), ngdbf.host_empty(F, np.int32), ngdbf.host_empty(F, np.uint8))
    yb = torch.from_numpy(y).pin_memory()
    outs_b = (torch.empty((F, nb), dtype=torch.uint8).pin_memory(), torch.empty(F, dtype=torch.int32).pin_memory(),
              torch.empty(F, dtype=torch.uint8).pin_memory())
    dc.decode_host(ya, sig, gp, seed=5, out=outs_a, chunk_frames=1024)
    dc.decode_host(yb, sig, gp, seed=5, out=outs_b, chunk_frames=1024)
    for a, b in zip(outs_a, outs_b):
        assert torch.equal(a, b)
    dc.close()


@pytest.mark.parametrize("mode", ["staged", "direct"])
@pytest.mark.parametrize("pinned", [True, False])
def test_decode_host_copy_modes_give_the_same_bits(mode, pinned):
    """Staged and direct copies, from page-locked and pageable buffers, decode the same frames
    bit for bit (small chunks, so that several staging pieces and chunks are in flight)."""
    code = wl.code_c2()
    F = 2500
    y, _, sig = wl.frames(code, F, 4.0, seed=78)
    dc = ngdbf.DeviceCode.from_code(code)
    gp = ngdbf.make_params(w=0.1875, theta=-0.7, eta=0.65, lam=0.993, y_max=2.0, t_max=300, variant=3)
    ref = dc.decode(torch.from_numpy(y).cuda(), sig, gp, seed=9)
    yin = torch.from_numpy(y).pin_memory() if pinned else torch.from_numpy(y.copy())
    old = ngdbf.ngdbf_get_host_copy_mode()
    try:
        ngdbf.ngdbf_set_host_copy_mode(ngdbf.NGDBF_HOST_COPY_STAGED if mode == "staged" else ngdbf.NGDBF_HOST_COPY_DIRECT)
        bits, iters, pas = dc.decode_host(yin, sig, gp, seed=9, chunk_frames=700)
    finally:
        ngdbf.ngdbf_set_host_copy_mode(old)
    assert np.array_equal(bits, ref[0].cpu().numpy())
    assert np.array_equal(iters, ref[1].cpu().numpy())
    assert np.array_equal(pas, ref[2].cpu().numpy())
    dc.close()


def test_concurrent_host_decodes_share_the_staging_pool():
    """Several threads call ngdbf_decode_host at once (staged copies: the library's staging
    buffers and host copy threads are shared); each result equals the device-buffer decode."""
    import threading
    code = wl.code_c1()
    gp = ngdbf.make_params(w=0.75, theta=-0.9, eta=0.96, y_max=2.5, t_max=100, variant=0)
    dc = ngdbf.DeviceCode.from_code(code)
    inputs = []
    for t in range(4):
        y, _, sig = wl.frames(code, 1500 + 300 * t, 3.75, seed=500 + t)
        inputs.append((y, sig))
    refs = []
    for t, (y, sig) in enumerate(inputs):
        b, i, p = dc.decode(torch.from_numpy(y).cuda(), sig, gp, seed=31, frame_offset=10 ** 6 * t)
        refs.append((b.cpu().numpy(), i.cpu().numpy(), p.cpu().numpy()))
    got = [None] * len(inputs)
    errors = []

    def run(t):
        try:
            torch.cuda.set_device(0)
            y, sig = inputs[t]
            got[t] = dc.decode_host(y, sig, gp, seed=31, frame_offset=10 ** 6 * t, chunk_frames=400)
        except Exception as e:          # reported below
            errors.append(e)

    ths = [threading.Thread(target=run, args=(t,)) for t in range(len(inputs))]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    assert not errors, errors
    for g, r in zip(got, refs):
        assert all(np.array_equal(a, b) for a, b in zip(g, r))
    dc.close()
