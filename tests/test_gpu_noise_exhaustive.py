"""The sampler's Box-Muller transform against the oracle's, bit for bit, over its
whole input domain.  Its two pieces each take a 24-bit integer: the radius
sqrt(-2 ln u1) of u1 = (i + 1) 2^-24 (the project-written FP32 ln, then a square
root), and cos, sin of 2 pi i 2^-24 (the quarter-turn reduction and the Taylor
polynomials).  Every one of the 2^24 inputs of each is computed on the device by
the code the sampling kernels run and compared with the oracle's C functions
(radius: the oracle's ln, then an IEEE single-precision square root).  A
normal is radius x cos or radius x sin, one correctly rounded product on both
sides, so this pins every normal the sampler can draw."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2409_10469_gb300 import _mppi  # noqa: E402

pytestmark = pytest.mark.gpu

N = 1 << 24


@pytest.fixture(scope="module")
def tables():
    import __graft_entry__ as g
    g.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    r = torch.empty(N, device="cuda")
    c = torch.empty(N, device="cuda")
    s = torch.empty(N, device="cuda")
    assert _mppi.lib().mppi_selftest_noise_tables(_mppi._ptr(r), _mppi._ptr(c), _mppi._ptr(s), None) == 0
    torch.cuda.synchronize()
    return r.cpu().numpy(), c.cpu().numpy(), s.cpu().numpy()


def test_radius_bit_exact_for_every_input(tables):
    r, _, _ = tables
    u1 = (np.arange(N, dtype=np.float64) + 1.0).astype(np.float32) * np.float32(2.0 ** -24)
    ro = np.sqrt(np.float32(-2.0) * O.lnf(u1)).astype(np.float32)
    bad = np.flatnonzero(r.view(np.uint32) != ro.view(np.uint32))
    assert bad.size == 0, (bad[:8], r[bad[:8]], ro[bad[:8]])


def test_sincos_bit_exact_for_every_input(tables):
    _, c, s = tables
    co, so = O.sincos_u24(np.arange(N, dtype=np.uint32))
    assert np.array_equal(c.view(np.uint32), co.view(np.uint32))
    assert np.array_equal(s.view(np.uint32), so.view(np.uint32))
