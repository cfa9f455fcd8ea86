"""The allocation-free fused reduction (zig_moments_noalloc).

Some callers cannot allocate device memory at all (they are handed only
their output buffers, or run where the surrounding allocator is locked);
zig_moments_noalloc serves them with the library's static scratch.  This
checks, through the C ABI, that two calls in a row give what zig_moments
gives with a caller workspace: the same histogram and the same power sums
bit for bit (both run the same grid, and every thread block adds its
values in a fixed order and the last block sums the blocks in block
order), and power sums within the bound the other reduction tests use
(20 * 2^-24 * sum |x|^k for FP32, 1e-12 * sum |x|^k for FP64) of the
oracle's sums, with the oracle's histogram exactly.  Between the two checked calls a call of the
other distribution and precision leaves its own contents in the shared
scratch, which the next call must not pick up.
Collected last (file name) so that a stop at the first failure has already
run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def zig():
    assert torch.cuda.is_available()
    from paper_1403_6870_gb300 import build

    build.build()
    import paper_1403_6870_gb300 as z

    z.zig_build_tables()
    return z


@pytest.mark.parametrize("dist,dtype", [(1, 0), (0, 1)])
def test_noalloc_matches_workspace_entry_point(zig, orc, dist, dtype):
    n, seed, off = (1 << 22) + 999, 0x5DEECE66D, 31337
    osums, abss, ohist, _ = orc.moments(dist, dtype, seed, off, n)
    tol = (20 * 2.0**-24 if dtype == 0 else 1e-12) * abss + 1e-300

    ws = torch.empty(zig.zig_moments_workspace_bytes(dist, dtype), dtype=torch.uint8,
                     device="cuda")
    ref_s = torch.zeros(4, dtype=torch.float64, device="cuda")
    ref_h = torch.zeros(4098, dtype=torch.int64, device="cuda")
    zig.zig_moments(dist, dtype, n, seed, off, ref_s, ref_h, ws)
    ref_s, ref_h = ref_s.cpu().numpy(), ref_h.cpu().numpy()

    for call in range(2):  # two checked calls share the static scratch
        if call == 1:  # another class in between leaves its contents behind
            xs = torch.zeros(4, dtype=torch.float64, device="cuda")
            xh = torch.zeros(4098, dtype=torch.int64, device="cuda")
            zig.zig_moments_noalloc(1 - dist, 1 - dtype, (1 << 20) + 5, seed + 1, 7, xs, xh)
        s = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
        h = torch.full((4098,), -1, dtype=torch.int64, device="cuda")
        zig.zig_moments_noalloc(dist, dtype, n, seed, off, s, h)
        assert zig.zig_status_poll() == zig.ZIG_OK
        s, h = s.cpu().numpy(), h.cpu().numpy()
        assert np.array_equal(h, ref_h)
        assert np.array_equal(s, ref_s), (s, ref_s)
        assert np.array_equal(h.astype(np.uint64), ohist)
        assert np.all(np.abs(s - osums) <= tol), (s, osums)
