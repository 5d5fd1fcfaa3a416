"""The decoder's perturbation generator against the reference decoder's, over every input.

Each Box-Muller output is fl32(rho(a0) * cos or sin(a1)) with a0, a1 the 23-bit
integers r >> 9 of two Philox outputs, so equality of rho and of (sin, cos) for all
2^23 values of a, together with the Philox known-answer and parity tests, covers
every perturbation either side can draw.
"""
import numpy as np
import pytest

import oracle
from paper_1402_2773_gb300 import ngdbf

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


def test_generator_factors_bit_exact_over_the_whole_domain():
    O = oracle.load()
    rho = torch.empty(1 << 23, dtype=torch.float32, device="cuda")
    sn = torch.empty_like(rho)
    cs = torch.empty_like(rho)
    ngdbf.ngdbf_generator_factors(rho.data_ptr(), sn.data_ptr(), cs.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    want_rho = O.rho_all()
    want_sn, want_cs = O.sincos_all()
    for got, want, name in ((rho, want_rho, "rho"), (sn, want_sn, "sin"), (cs, want_cs, "cos")):
        g = got.cpu().numpy().view(np.uint32)
        w = want.view(np.uint32)
        bad = np.nonzero(g != w)[0]
        assert bad.size == 0, f"{name}: {bad.size} of 2^23 values differ, first a = {bad[:5]}"
