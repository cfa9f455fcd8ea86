"""CPU checks of the library's per-box shortcut bounds of the overhang test
(zig_tables_ex acc52/rej52/acc23/rej23: the per-overhang eps of Appendix D
item 2 and the normal's convex/concave regions).

The bounds only let the device skip the exact test y < P(x); they must
never change its answer.  For boxes at both index widths and several ux,
the point just inside each bound is given to the oracle: its exact FP64
test (orc_overhang_attempt64) and its FP32 sampler (scripted words) must
accept below acc and reject above rej.  The share of attempts that still
need the exact test is compared with the single-eps rule.
"""
import numpy as np
import pytest

pytestmark = []

ONE52, ONE23 = 1 << 52, 1 << 23


@pytest.fixture(scope="module")
def zig():
    from paper_1403_6870_gb300 import build

    build.build()
    import paper_1403_6870_gb300 as z

    return z


def _alias_word(t, j):
    K = 1 << t.abits
    if int(t.T[j]) > 0:
        return j
    for c in range(t.imax):
        if int(t.alias[c]) == j and int(t.T[c]) < K:
            return c | ((K - 1) << (64 - t.abits))
    raise AssertionError("no column reaches j")


def _boxes(L, width):
    js = list(range(1, L + 1)) if width == 8 else sorted(set(
        list(range(1, 9)) + list(range(1, L + 1, 37)) + list(range(L - 8, L + 1))))
    return js


@pytest.mark.parametrize("width", [8, 10])
@pytest.mark.parametrize("dist", [0, 1])
def test_bounds_agree_with_the_exact_test(zig, orc, dist, width):
    lib = zig.zig_export_tables_ex(dist, width)
    t = orc.tables(dist, width, 52, 64 - width)
    te, tn = orc.tables(0, width, 52, 64 - width), orc.tables(1, width, 52, 64 - width)
    L = t.L
    fringe_i = L  # a layer index at or above L_max
    checked = 0
    for j in _boxes(L, width):
        acc, rej = int(lib.acc52[j]), int(lib.rej52[j])
        acc32, rej32 = int(lib.acc23[j]), int(lib.rej23[j])
        assert 0 <= acc <= ONE52 and rej >= ONE52 and 0 <= acc32 <= ONE23 and rej32 >= ONE23
        for f in (0.0, 0.013, 0.25, 0.5, 0.77, 0.999):
            # FP64: the oracle's exact test
            mx = int(f * ONE52)
            my = acc - 1 - mx
            if acc > 0 and 0 <= my < ONE52:
                ok, _ = orc.overhang_attempt(t, j, mx / ONE52, my / ONE52)
                assert ok, (dist, width, j, f, "acc52")
                checked += 1
            my = rej + 1 - mx
            if dist == 1 and 0 <= my < ONE52:
                ok, _ = orc.overhang_attempt(t, j, mx / ONE52, my / ONE52)
                assert not ok, (dist, width, j, f, "rej52")
                checked += 1
            # FP32: the oracle's FP32 sampler on scripted words (accept after
            # three words; a rejection asks for more and overruns the script)
            mx = int(f * ONE23)
            for my, want in ((acc32 - 1 - mx, True), (rej32 + 1 - mx, False)):
                if not 0 <= my < ONE23 or (want and acc32 == 0) or (not want and dist == 0):
                    continue
                w0 = fringe_i | (mx << 41)
                words = [w0, _alias_word(t, j), my << 41]
                x, used, overrun, err = orc.sample_script(dist, words, orc.F32, te=te, tn=tn)
                assert (not overrun and used == 3) == want, (dist, width, j, f, want)
                checked += 1
    assert checked > 100


@pytest.mark.parametrize("dist", [0, 1])
def test_exact_test_rate(zig, orc, dist):
    """Share of first attempts (box j with probability A_j / sum A) that
    still need the exact test, FP64, single-eps rule against per-box bounds."""
    lib = zig.zig_export_tables_ex(dist, 8)
    t = orc.tables(dist)
    rng = np.random.default_rng(5)
    A = np.array([t.A[j] for j in range(1, t.L + 1)])
    w = A / A.sum()
    old = new = 0.0
    tau52 = int(np.ceil(t.tau * ONE52)) if dist == 0 else 0
    for j in range(1, t.L + 1):
        mx = rng.integers(0, ONE52, 4000, dtype=np.int64).astype(object)
        my = rng.integers(0, ONE52, 4000, dtype=np.int64).astype(object)
        s = np.array([a + b for a, b in zip(mx, my)], dtype=object)
        if dist == 0:
            s = np.where(s > ONE52, 2 * ONE52 - s, s)  # reflection
            need_old = s >= tau52
        else:
            need_old = np.ones(len(s), dtype=bool)
        need_new = (s >= int(lib.acc52[j])) & (s <= int(lib.rej52[j]))
        old += w[j - 1] * float(np.mean(need_old))
        new += w[j - 1] * float(np.mean(need_new))
    assert new <= old
    # the per-box bounds remove most of the exact tests
    assert new < (0.6 if dist == 0 else 0.25) * old, (old, new)
