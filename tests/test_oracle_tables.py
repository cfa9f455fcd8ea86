"""Pins for the oracle's tables (Sec. 2 of arXiv:1403.6870).

Each check compares the oracle's binary128-built, binary64-rounded tables
with something fixed independently of its code: the paper's printed L_max,
the Lambert-W closed form of the exponential tail point, 40-digit mpmath
evaluations of the defining equations, numerical quadrature of the overhang
integrals, brute-force maximisation of the chord gap, and exact integer
identities of the alias table.  The structural pins run at both index
widths: 8 bits (i_max = 256, the paper's tables) and 10 bits (i_max = 1024,
the variant of Appendix D item 1).
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

mp = pytest.importorskip("mpmath")
mp.mp.dps = 40

IMAX = 256
# (index bits, alias threshold bits) of the two widths the library builds
WIDTHS = [(8, 56), (10, 54)]


def _P(dist, x):
    """Normalised density on x >= 0 (mpmath)."""
    x = mp.mpf(x)
    if dist == 0:
        return mp.e ** (-x)
    return mp.sqrt(2 / mp.pi) * mp.e ** (-x * x / 2)


def _ulp(x):
    return math.ulp(abs(x)) if x != 0 else math.ulp(0.0)


@pytest.fixture(scope="module")
def te(orc):
    return orc.tables(orc.EXP)


@pytest.fixture(scope="module")
def tn(orc):
    return orc.tables(orc.NORMAL)


def test_L_max_exponential_matches_paper(te):
    # Sec. 2: "for an exponential distribution L_max = 252 when i_max = 256".
    assert te.imax == 256 and te.L == 252


def test_L_max_normal_and_exit_rates(tn, te):
    # No printed value for the normal; 253 layers fit (fringe 3/256 = 1.17%,
    # within the paper's "<2% of cases" of Fig. 1's caption).
    assert tn.L == 253
    assert (IMAX - te.L) / IMAX == pytest.approx(0.015625)  # "4/256 = 1.6%"
    assert (IMAX - tn.L) / IMAX < 0.02


def test_tail_point_exponential_lambert_w(te):
    # X_0 e^{-X_0} = 1/256 on the larger branch: X_0 = -W_{-1}(-1/256).
    x0 = -special.lambertw(-1.0 / 256, k=-1).real
    assert abs(te.X[0] - x0) <= 2 * _ulp(x0)
    assert te.X[0] == pytest.approx(7.5692746941480624, rel=1e-15)


def test_tail_point_normal_root(tn):
    x0 = mp.findroot(lambda x: x * _P(1, x) - mp.mpf(1) / 256, 3.6)
    assert abs(tn.X[0] - float(x0)) <= _ulp(float(x0))


@pytest.mark.parametrize("width", WIDTHS)
@pytest.mark.parametrize("dist", [0, 1])
def test_layers_equal_area_residuals(orc, dist, width):
    t = orc.tables(dist, width[0], 52, width[1])
    IMAX = t.imax
    fprev = mp.mpf(0)
    Xprev = None
    for k in range(t.L):
        X = mp.mpf(t.X[k])
        fk = _P(dist, X)
        res = X * (fk - fprev) - mp.mpf(1) / IMAX
        # The residual with binary64 abscissae is bounded by the rounding of
        # X_k and X_{k-1} times the partial derivatives of the area.
        dX = abs(fk * (1 - X) - fprev) if dist == 0 else abs(fk * (1 - X * X) - fprev)
        bound = dX * _ulp(t.X[k]) + (X * abs(_P(dist, Xprev) * (Xprev if dist == 0 else Xprev ** 2)) * _ulp(float(Xprev)) if Xprev is not None else 0)
        assert abs(res) <= 2 * bound + mp.mpf(10) ** -30, (k, float(res))
        # Larger root: the area decreases in X there (Sec. 2, read R1).
        slope = (fk * (1 - X) - fprev) if dist == 0 else (fk * (1 - X * X) - fprev)
        assert slope < 0, k
        # Stored heights are the (unnormalised for the normal) density.
        # f_k was rounded from the binary128 abscissa, so allow the slope of
        # the density times half an ulp of X_k on top of the final rounding.
        h = mp.e ** (-X) if dist == 0 else mp.e ** (-X * X / 2)
        dh = h if dist == 0 else h * X
        assert abs(t.f[k] - h) <= _ulp(float(h)) + dh * _ulp(t.X[k]) / 2, k
        fprev, Xprev = fk, X
    # No further layer of area 1/i_max fits above the last one: max_X of
    # X (P(X) - f_{L-1}) over [0, X_{L-1}] is below 1/i_max.
    xs = np.linspace(0, t.X[t.L - 1], 20001)
    g = max(float(mp.mpf(x) * (_P(dist, x) - fprev)) for x in xs[::50])
    assert g < 1.0 / IMAX
    assert t.X[t.L] == 0.0 and t.f[t.L] == 1.0


@pytest.mark.parametrize("width", WIDTHS)
@pytest.mark.parametrize("dist", [0, 1])
def test_differences(orc, dist, width):
    t = orc.tables(dist, width[0], 52, width[1])
    for j in range(1, t.L + 1):
        ref_dx = t.X[j - 1] - t.X[j]
        assert abs(t.dX[j] - ref_dx) <= _ulp(t.X[j - 1]) + _ulp(t.X[j]) + _ulp(ref_dx), j
        ref_df = t.f[j] - t.f[j - 1]
        assert abs(t.df[j] - ref_df) <= _ulp(t.f[j - 1]) + _ulp(t.f[j]) + _ulp(ref_df), j
        assert t.dX[j] > 0 and t.df[j] > 0


@pytest.mark.parametrize("width", WIDTHS)
@pytest.mark.parametrize("dist", [0, 1])
def test_overhang_masses_quadrature(orc, dist, width):
    t = orc.tables(dist, width[0], 52, width[1])
    c = math.sqrt(2 / math.pi)
    dens = (lambda x: math.exp(-x)) if dist == 0 else (lambda x: c * math.exp(-x * x / 2))
    fn = [dens(t.X[k]) for k in range(t.L)] + [dens(0.0)]
    for j in range(1, t.L + 1):
        a, b = t.X[j], t.X[j - 1]
        val, err = integrate.quad(lambda x: dens(x) - fn[j - 1], a, b, epsabs=1e-18, epsrel=1e-12)
        assert t.A[j] == pytest.approx(val, rel=1e-8, abs=1e-16), j
    tail = math.exp(-t.X[0]) if dist == 0 else special.erfc(t.X[0] / math.sqrt(2))
    assert t.A[0] == pytest.approx(tail, rel=1e-13)


@pytest.mark.parametrize("width", WIDTHS)
@pytest.mark.parametrize("dist", [0, 1])
def test_total_mass_is_one(orc, dist, width):
    t = orc.tables(dist, width[0], 52, width[1])
    total = mp.mpf(t.L) / t.imax + mp.fsum(mp.mpf(t.A[j]) for j in range(t.L + 1))
    assert abs(total - 1) < 1e-15
    # The cap above the last layer carries real mass (read R2).
    assert t.A[t.L] > 1e-3


def test_epsilon_bruteforce(te):
    eps = np.zeros(te.L + 1)
    for j in range(1, te.L + 1):
        x = np.linspace(te.X[j], te.X[j - 1], 200001)
        fj, fj1 = math.exp(-te.X[j]), math.exp(-te.X[j - 1])
        chord = fj + (x - te.X[j]) * (fj1 - fj) / (te.X[j - 1] - te.X[j])
        eps[j] = np.max(chord - np.exp(-x)) / (fj - fj1)
        assert te.eps_j[j] == pytest.approx(eps[j], rel=1e-6, abs=1e-12), j
        assert te.eps_j[j] > 0
    # Sec. 2: "the widest narrow band is still only 9% of the box height".
    assert int(np.argmax(eps)) == 1
    assert 0.09 <= te.eps <= 0.095
    assert te.eps == pytest.approx(eps.max(), rel=1e-6)
    # tau = RD(1 - eps (1 + 2^-40)) sits just below 1 - eps.
    assert te.tau < 1 - te.eps and te.tau > 1 - te.eps - 1e-11


@pytest.mark.parametrize("width", WIDTHS)
@pytest.mark.parametrize("dist", [0, 1])
def test_alias_reconstruction_identity(orc, dist, width):
    t = orc.tables(dist, width[0], 52, width[1])
    IMAX = t.imax
    K = 1 << t.abits
    q = [int(v) for v in t.q][:IMAX]
    T = [int(v) for v in t.T][:IMAX]
    al = [int(v) for v in t.alias][:IMAX]
    assert sum(q) == IMAX * K
    assert all(0 <= T[c] <= K for c in range(IMAX))
    rec = [0] * IMAX
    for c in range(IMAX):
        rec[c] += T[c]
        if al[c] != c:
            rec[al[c]] += K - T[c]
        else:
            assert T[c] == K
    assert rec == q
    # Integer weights follow the masses: q_j = RN(A_j / sum A * 2^64), with
    # the rounding residual on the largest weight only.
    A = [mp.mpf(t.A[j]) for j in range(t.L + 1)]
    s = mp.fsum(A)
    big = int(np.argmax(q))
    for j in range(IMAX):
        ideal = A[j] / s * IMAX * K if j <= t.L else 0
        tol = 3 + (2 ** 20 if j == big else 0) + float(abs(ideal)) * 1e-15
        assert abs(q[j] - ideal) <= tol, j
    assert all(q[j] == 0 for j in range(t.L + 1, IMAX))


def test_alias_pick_frequencies(orc, te):
    rng = np.random.default_rng(7)
    n = 1 << 18
    words = rng.integers(0, 2**63, size=n, dtype=np.uint64) * np.uint64(2) + \
        rng.integers(0, 2, size=n, dtype=np.uint64)
    js = np.array([orc.alias_pick(te, int(w)) for w in words])
    counts = np.bincount(js, minlength=IMAX)
    p = np.array([int(v) for v in te.q][:IMAX], dtype=float) / 2.0**64
    m = p > 0
    assert counts[~m].sum() == 0
    chi2 = float(((counts[m] - n * p[m]) ** 2 / (n * p[m])).sum())
    df = int(m.sum()) - 1
    assert chi2 < df + 6 * math.sqrt(2 * df)


@pytest.mark.parametrize("width", WIDTHS)
def test_fp32_tables_are_roundings(orc, width):
    for dist in (0, 1):
        t = orc.tables(dist, width[0], 52, width[1])
        for k in range(t.L + 1):
            assert abs(float(t.X32[k]) - t.X[k]) <= np.spacing(np.float32(abs(t.X[k]))) / 2 * (1 + 1e-6)
            assert abs(float(t.f32[k]) - t.f[k]) <= np.spacing(np.float32(abs(t.f[k]))) / 2 * (1 + 1e-6)
        assert float(t.rinv32) == pytest.approx(1 / t.X[0], rel=2**-24)
        assert t.rinv == pytest.approx(1 / t.X[0], rel=2**-52)


def test_reduced_width_tables(orc):
    """imax = 8 tables: same construction, mass identity, exact alias."""
    for dist in (0, 1):
        t = orc.tables(dist, 3, 12, 12)
        assert t.imax == 8 and 1 <= t.L < 8
        total = t.L / 8 + sum(t.A[j] for j in range(t.L + 1))
        assert total == pytest.approx(1.0, abs=1e-14)
        assert sum(int(v) for v in list(t.q)[:8]) == 8 << 12


def test_ten_bit_tables_epsilon_and_layers(orc):
    """i_max = 1024: the chord deviation by brute force (as for 256), and
    the layer counts and tail points move the way the construction says
    (more, thinner layers; a tail point further out)."""
    te = orc.tables(0, 10, 52, 54)
    tn = orc.tables(1, 10, 52, 54)
    for j in (1, 2, 100, te.L // 2, te.L):
        x = np.linspace(te.X[j], te.X[j - 1], 200001)
        fj, fj1 = math.exp(-te.X[j]), math.exp(-te.X[j - 1])
        chord = fj + (x - te.X[j]) * (fj1 - fj) / (te.X[j - 1] - te.X[j])
        assert te.eps_j[j] == pytest.approx(np.max(chord - np.exp(-x)) / (fj - fj1), rel=1e-6)
    assert te.eps == pytest.approx(max(te.eps_j[j] for j in range(1, te.L + 1)))
    # X_0 solves X e^-X = 1/1024 (larger root): -W_{-1}(-1/1024)
    x0 = -mp.lambertw(-mp.mpf(1) / 1024, -1)
    assert abs(te.X[0] - float(x0)) <= 2 * _ulp(float(x0))
    t8e, t8n = orc.tables(0), orc.tables(1)
    assert te.L > 4 * t8e.L - 8 and tn.L > 4 * t8n.L - 8
    assert te.X[0] > t8e.X[0] and tn.X[0] > t8n.X[0]
