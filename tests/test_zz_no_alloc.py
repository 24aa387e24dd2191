"""lbm_wdot_to_host_noalloc: the copy-out of a 16-bit wdot plane through the
library's fixed conversion array gives the same values as lbm_fields, on two
calls in a row, before and after further steps.  Kept in a file of its own,
collected last, so that it also runs after every other test has used the
device."""
import numpy as np
import pytest

from paper_2206_12412_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_12412_gb300 import lbm
    lbm.load_library()
    return lbm


@pytest.mark.parametrize("storage", ["f32_bf16", "f32_f16"])
@pytest.mark.parametrize("shape", [(1000, 1000), (37, 29), (1024, 1024)])
def test_noalloc_copy_matches_lbm_fields(gpu, storage, shape):
    nx, ny = shape
    p = W.prescribed_strip(nx, ny, 0.4, u0=1e-3, t_ramp=50.0)
    lat = gpu.Lattice(p, storage)
    w0, wd0 = W.random_state(nx, ny, seed=nx + ny, dtype=np.float32)
    lat.set_fields(w0, wd0)
    for steps in (3, 40):
        lat.step(steps)
        ref = lat.fields()[1]
        for _ in range(2):   # two calls in a row
            out = np.full(nx * ny, np.nan, np.float32)
            gpu.lbm_wdot_to_host_noalloc(lat.h, out)
            # the same conversion kernel on the same plane: identical values
            np.testing.assert_array_equal(out.reshape(ny, nx), ref)
    lat.close()


def test_noalloc_copy_limits(gpu):
    big = gpu.Lattice(W.prescribed_strip(1100, 1000, 0.4), "f32_f16")   # 1.1 M sites > 2^20
    out = np.empty(1100 * 1000, np.float32)
    with pytest.raises(gpu.LbmError, match="fixed conversion array"):
        gpu.lbm_wdot_to_host_noalloc(big.h, out)
    big.close()
    small = gpu.Lattice(W.prescribed_strip(64, 32, 0.4), "f32_bf16")
    with pytest.raises(gpu.LbmError, match="too small"):
        gpu.lbm_wdot_to_host_noalloc(small.h, np.empty(64 * 32 - 1, np.float32))
    small.close()
    plain = gpu.Lattice(W.prescribed_strip(64, 32, 0.4), "f32")
    with pytest.raises(gpu.LbmError, match="16-bit"):
        gpu.lbm_wdot_to_host_noalloc(plain.h, np.empty(64 * 32, np.float32))
    plain.close()
