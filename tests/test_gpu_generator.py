"""The decoder's perturbation generator against the reference decoder's, over every input.

Each perturbation is fl32(eta sigma) * z(r) with r one Philox output and z the
inverse-CDF deviate of r, so equality of z(r) for all 2^32 values of r, together
with the Philox known-answer and decode parity tests, covers every perturbation
either side can draw.
"""
from concurrent.futures import ThreadPoolExecutor
import os

import numpy as np
import pytest

import oracle
from paper_1402_2773_gb300 import ngdbf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
CHUNK = 1 << 27
THREADS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_2773_gb300 import _build
    _build.build_cuda()
    ngdbf.load()
    torch.cuda.set_device(0)


def test_deviates_bit_exact_over_every_philox_output():
    O = oracle.load()
    buf = torch.empty(CHUNK, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    part = CHUNK // THREADS
    with ThreadPoolExecutor(THREADS) as pool:
        for c in range((1 << 32) // CHUNK):
            start = c * CHUNK
            ngdbf.ngdbf_gaussian_range(start, CHUNK, buf.data_ptr(), stream)
            want = np.concatenate(list(pool.map(lambda i: O.gauss_range_f32(start + i * part, part),
                                                range(THREADS))))
            got = buf.cpu().numpy()
            bad = np.nonzero(got.view(np.uint32) != want.view(np.uint32))[0]
            assert bad.size == 0, f"{bad.size} deviates differ in chunk {c}, first r = {start + bad[:4]}"


def test_zero_count_and_host_buffer():
    ngdbf.ngdbf_gaussian_range(5, 0, 0)
    host = np.zeros(4, np.float32)
    with pytest.raises(RuntimeError):
        ngdbf.ngdbf_gaussian_range(0, 4, host.ctypes.data)
