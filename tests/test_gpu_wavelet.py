"""GPU parity of the periodised Daubechies-4 transform W and W^H (Sec. 2, Sec. 6) against the
oracle; tolerance 1e-6 relative l2 (8-tap float32 filters per level)."""
import numpy as np
import pytest

from oracle import wavelet as owv
from tests.gpu_util import need_gpu, rel, to_dev, make_plan

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape,levels", [((256, 256), 4), ((48, 80), 3), ((32, 16, 24), 3), ((16, 16), 4)])
def test_dwt_roundtrip(shape, levels):
    need_gpu()
    rng = np.random.default_rng(sum(shape))
    x = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)
    ref = owv.dwt(x.astype(np.complex128), levels)
    plan = make_plan(shape, 1, 16, 1.25, levels)
    c = plan.wavelet(to_dev(x), forward=True)
    assert rel(c.cpu().numpy(), ref) < 1e-6
    xi = plan.wavelet(to_dev(ref.astype(np.complex64)), forward=False).cpu().numpy()
    assert rel(xi, owv.idwt(ref, levels)) < 1e-6
