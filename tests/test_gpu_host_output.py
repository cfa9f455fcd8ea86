"""GPU: outputs in page-locked host memory.

zig_normal / zig_exponential / zig_generate write page-locked host memory
(torch pin_memory, i.e. cudaHostAlloc) directly through its device alias;
the bits equal those written to device memory for the same counters,
including misaligned views and ragged sizes.  Pageable host memory is
refused before any launch.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def zig():
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    from paper_1403_6870_gb300 import build

    build.build()
    import paper_1403_6870_gb300 as z

    z.zig_build_tables()
    return z


@pytest.mark.parametrize("dist", [W.EXP, W.NORMAL])
@pytest.mark.parametrize("dtype", [W.F64, W.F32])
@pytest.mark.parametrize("pad", [0, 3])
def test_pinned_host_output_equals_device_output(zig, dist, dtype, pad):
    n = (1 << 20) + 4099
    tdt = torch.float64 if dtype == W.F64 else torch.float32
    dev = torch.empty(n, dtype=tdt, device="cuda")
    host = torch.full((n + pad + 8,), float("nan"), dtype=tdt).pin_memory()
    view = host[pad:pad + n]
    fn = zig.zig_exponential if dist == W.EXP else zig.zig_normal
    fn(dev, n, 77, 2**32 - 1000)
    fn(view, n, 77, 2**32 - 1000)
    torch.cuda.synchronize()
    it = np.uint64 if dtype == W.F64 else np.uint32
    assert np.array_equal(view.numpy().view(it), dev.cpu().numpy().view(it))
    h = host.numpy()
    assert np.all(np.isnan(h[:pad])) and np.all(np.isnan(h[pad + n:]))
    # packed keying through zig_generate as well
    zig.zig_generate(dist, 1, dev, n, 5, 8)
    zig.zig_generate(dist, 1, view, n, 5, 8)
    torch.cuda.synchronize()
    assert np.array_equal(view.numpy().view(it), dev.cpu().numpy().view(it))
    assert zig.zig_status_poll() == zig.ZIG_OK


def test_pageable_host_memory_is_refused(zig):
    a = np.zeros(1024, dtype=np.float64)  # ordinary (pageable) host memory
    st = zig.raw_call("zig_normal", a.ctypes.data, 1024, 1, 0, zig.ZIG_F64, None)
    assert st == zig.ZIG_E_INVAL
    assert np.all(a == 0.0)
    with pytest.raises(ValueError):
        zig.zig_normal(torch.zeros(16, dtype=torch.float64), 16, 1, 0)
