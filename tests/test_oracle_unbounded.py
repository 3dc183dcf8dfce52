"""Pins for the oracle's unbounded solve (Sec. 2.6, Hockney-Eastwood) and G2 kernel.

  * brute-force direct summation psi_i = -s h^d sum_j G(x_i - x_j) f_j on
    small grids (the exact result the doubled-domain convolution must equal);
  * the kernel itself: -lap G = Gaussian checked by finite differences of the
    closed form, and the r -> 0 limits;
  * the Gaussian semigroup closed form of a blob's potential,
    erf(r / sqrt(2(s^2 + sigma^2))) / (4 pi r) in 3D, with the error falling
    as the grid is refined;
  * the curl: the doubled-domain solution differentiated in real space with
    the closed-form Fourier differentiation matrix.
"""
import math

import numpy as np
import pytest
from scipy import special

import oracle
import workloads
from oracle import green
from oracle.desc import Desc


def direct_sum(desc, f, pts=None, padded=False):
    dim = desc.dim
    h = [desc.h(a) for a in range(dim)]
    n = [desc.n[a] for a in range(dim)]
    src = np.argwhere(np.ones(tuple(reversed(n)), dtype=bool))  # [j][(z),y,x]
    fv = f.reshape(-1)
    if pts is None:
        shape = tuple(2 * m for m in reversed(n)) if padded else tuple(reversed(n))
        pts = np.argwhere(np.ones(shape, dtype=bool))
    out = np.zeros(len(pts))
    hd = np.prod(h)
    for i, p in enumerate(pts):
        r2 = 0.0
        for k in range(dim):
            ax = dim - 1 - k
            d = p[k] - src[:, k]
            if padded:
                M = 2 * n[ax]
                d = np.mod(d, M)
                d = np.minimum(d, M - d)
            r2 = r2 + (d * h[ax]) ** 2
        out[i] = -desc.rhs_scale * hd * np.sum(green.green(dim, np.sqrt(r2), desc.sigma) * fv)
    return out


@pytest.mark.parametrize("dim,n", [(3, 6), (3, 8), (2, 12), (2, 16)])
def test_direct_sum(dim, n):
    rng = np.random.default_rng(n + dim)
    d = Desc(dim, (n, n + 2, n)[:dim], (-0.5,) * dim, (0.5, 0.7, 0.4)[:dim], ("U",) * dim, True,
             rhs_scale=-1.3, sigma=0.09)
    f = rng.normal(size=d.shape())
    psi, _ = oracle.solve(d, f)
    ref = direct_sum(d, f).reshape(d.shape())
    assert np.max(np.abs(psi[0] - ref)) < 1e-12 * np.max(np.abs(ref))


def test_kernel_laplacian_3d():
    sigma = 0.1
    eps = 1e-3
    for r in (0.03, 0.1, 0.25, 0.6):
        # radial Laplacian (1/r^2) d/dr (r^2 dG/dr) by central differences
        g = lambda s: green.g2_3d(np.array(s), sigma)
        d1p = (g(r + eps) - g(r)) / eps
        d1m = (g(r) - g(r - eps)) / eps
        lap = ((r + eps / 2) ** 2 * d1p - (r - eps / 2) ** 2 * d1m) / eps / r ** 2
        zeta = math.exp(-r * r / (2 * sigma * sigma)) / ((2 * math.pi) ** 1.5 * sigma ** 3)
        assert abs(lap + zeta) < 2e-4 * max(zeta, 1.0)


def test_kernel_laplacian_2d():
    sigma = 0.1
    eps = 1e-3
    for r in (0.03, 0.1, 0.25, 0.6):
        g = lambda s: green.g2_2d(np.array(s), sigma)
        d1p = (g(r + eps) - g(r)) / eps
        d1m = (g(r) - g(r - eps)) / eps
        lap = ((r + eps / 2) * d1p - (r - eps / 2) * d1m) / eps / r
        zeta = math.exp(-r * r / (2 * sigma * sigma)) / (2 * math.pi * sigma ** 2)
        assert abs(lap + zeta) < 2e-4 * max(zeta, 1.0)


def test_kernel_origin_limits():
    for sigma in (0.05, 0.3):
        r = np.array([1e-6 * sigma])
        assert abs(green.g2_3d(r, sigma)[0] - green.g2_3d(np.array([0.0]), sigma)[0]) < 1e-9
        assert abs(green.g2_2d(r, sigma)[0] - green.g2_2d(np.array([0.0]), sigma)[0]) < 1e-9


def blob_potential(r, s, sigma):
    a = math.sqrt(2 * (s * s + sigma * sigma))
    safe = np.where(r > 0, r, 1.0)
    return np.where(r > 0, special.erf(safe / a) / (4 * math.pi * safe), 2 / (a * 4 * math.pi ** 1.5))


def test_gaussian_blob_closed_form():
    errs = []
    for n in (24, 48):
        h = 1.0 / n
        sigma = 2 * h
        s = 0.06
        d = Desc(3, (n,) * 3, (-0.5,) * 3, (0.5,) * 3, ("U",) * 3, True, rhs_scale=-1.0, sigma=sigma)
        c = (0.5 * h, 0.5 * h, 0.5 * h)  # centred on a grid node
        f = workloads.gaussian_blob_field(n, c, s)
        psi, _ = oracle.solve(d, f)
        x = workloads.node_positions(-0.5, 0.5, n, True, n)
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        r = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2)
        ref = blob_potential(r, s, sigma)
        errs.append(np.max(np.abs(psi[0] - ref)) / np.max(ref))
    assert errs[1] < errs[0]
    assert errs[1] < 1e-3


def fourier_diff_matrix(M, period):
    """Trefethen's closed-form spectral differentiation matrix (Nyquist-free)."""
    D = np.zeros((M, M))
    for i in range(M):
        for j in range(M):
            if i == j:
                continue
            k = i - j
            if M % 2 == 0:
                D[i, j] = 0.5 * (-1) ** k / math.tan(k * math.pi / M)
            else:
                D[i, j] = 0.5 * (-1) ** k / math.sin(k * math.pi / M)
    return D * (2 * math.pi / period)


def test_curl_matches_real_space_differentiation():
    n = 6
    d = Desc(3, (n,) * 3, (-0.5,) * 3, (0.5,) * 3, ("U",) * 3, True, op="CURL", ncomp=3,
             rhs_scale=-1.0, sigma=0.15)
    rng = np.random.default_rng(5)
    f = rng.normal(size=(3, n, n, n))
    psi, u = oracle.solve(d, f)
    # full doubled-domain potential by brute force, then real-space derivatives
    full = np.stack([direct_sum(d, f[c], padded=True).reshape((2 * n,) * 3) for c in range(3)])
    Dm = fourier_diff_matrix(2 * n, 2 * n * d.h(0))
    dx = lambda a: np.einsum("ij,zyj->zyi", Dm, a)
    dy = lambda a: np.einsum("ij,zjx->zix", Dm, a)
    dz = lambda a: np.einsum("ij,jyx->iyx", Dm, a)
    curl = np.stack([dy(full[2]) - dz(full[1]), dz(full[0]) - dx(full[2]), dx(full[1]) - dy(full[0])])
    ref = curl[:, :n, :n, :n]
    np.testing.assert_allclose(psi, full[:, :n, :n, :n], atol=1e-12)
    assert np.max(np.abs(u - ref)) < 1e-11 * np.max(np.abs(ref))


def test_nabla_returns_source_ps_periodic():
    # NABLA after a PS solve gives back the source (minus its mean)
    n = 16
    d = Desc(3, (n,) * 3, (0,) * 3, (1.0, 2.0, 1.5), ("P",) * 3, True, "PS", op="NABLA")
    rng = np.random.default_rng(1)
    f = rng.normal(size=d.shape())
    _, lap = oracle.solve(d, f)
    np.testing.assert_allclose(lap[0], f - f.mean(), atol=1e-11)


@pytest.mark.parametrize("op,ncomp,dim", [("CURL", 3, 3), ("GRAD", 1, 3), ("DIV", 3, 3), ("CURL", 1, 2),
                                          ("NONE", 2, 3)])
def test_sampled_points_match_full_oracle(op, ncomp, dim):
    # the point-wise evaluation used at full size equals the full doubled-domain solve
    from oracle import unbounded
    n = (10, 8, 6)[:dim]
    d = Desc(dim, n, (-0.5,) * dim, (0.5, 0.4, 0.3)[:dim], ("U",) * dim, True, op=op, ncomp=ncomp,
             rhs_scale=-1.0, sigma=0.12)
    rng = np.random.default_rng(9)
    f = rng.normal(size=(ncomp,) + d.shape())
    psi, opo = oracle.solve(d, f)
    pts = [tuple(rng.integers(0, n[a]) for a in range(dim)) for _ in range(6)] + [tuple(0 for _ in n),
                                                                                 tuple(m - 1 for m in n)]
    ps, os_ = unbounded.sample_points(d, f, pts)
    for i, p in enumerate(pts):
        idx = tuple(reversed(p))
        np.testing.assert_allclose(ps[i], psi[(slice(None),) + idx], rtol=1e-11, atol=1e-13)
        if opo is not None:
            np.testing.assert_allclose(os_[i], opo[(slice(None),) + idx], rtol=1e-10, atol=1e-12)


# ---------------------------------------------------------------------------
# higher-order Gaussian kernels G4..G10 (Sec. 2.6.2)
# ---------------------------------------------------------------------------
def _zeta_fourier(dim, P, sigma, r):
    """zeta_P at radius r from its transform exp(-(k s)^2/2) sum_{j<P/2} (k s)^{2j}/(2^j j!) (radial quadrature)."""
    from scipy import integrate, special
    m = P // 2

    def zhat(k):
        return math.exp(-(k * sigma) ** 2 / 2) * sum((k * sigma) ** (2 * j) / (2 ** j * math.factorial(j)) for j in range(m))

    if dim == 3:
        return integrate.quad(lambda k: zhat(k) * k * math.sin(k * r), 0, 60 / sigma, limit=400)[0] / (2 * math.pi ** 2 * r)
    return integrate.quad(lambda k: zhat(k) * k * special.j0(k * r), 0, 60 / sigma, limit=400)[0] / (2 * math.pi)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("P", [2, 4, 6, 8, 10])
def test_higher_order_kernel_laplacian_is_fourier_smoothing(dim, P):
    # -lap G_P (finite differences of the closed form) equals the smoothing of order P
    # defined in Fourier space, computed independently by quadrature
    sig = 0.7
    scale = abs(_zeta_fourier(dim, P, sig, 1e-3))
    for r in (0.2, 0.7, 1.3, 2.5):
        d = 1e-3
        g = lambda x: float(green.green(dim, np.array(x), sig, f"G{P}"))
        g0, gp, gm = g(r), g(r + d), g(r - d)
        lap = (gp - 2 * g0 + gm) / d ** 2 + (dim - 1) / r * (gp - gm) / (2 * d)
        assert abs(-lap - _zeta_fourier(dim, P, sig, r)) < 1e-4 * scale


def test_higher_order_kernels_converge_faster_on_a_blob():
    # Gaussian blob of width s: the unregularised potential is erf(r/(s sqrt 2))/(4 pi r);
    # at sigma = 2h the solve's error falls with every step of the kernel order
    from scipy import special
    n = 32
    h = 1.0 / n
    x = -0.5 + h * (np.arange(n) + 0.5)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    R = np.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    s = 0.08
    om = np.exp(-R ** 2 / (2 * s * s)) / (2 * math.pi * s * s) ** 1.5
    exact = special.erf(R / (math.sqrt(2) * s)) / (4 * math.pi * R)
    errs = []
    for P in (2, 4, 6, 8, 10):
        d = Desc(3, (n,) * 3, (-0.5,) * 3, (0.5,) * 3, ("U",) * 3, True, rhs_scale=-1.0, sigma=2 * h, kernel=f"G{P}")
        psi, _ = oracle.solve(d, om[None])
        errs.append(np.max(np.abs(psi[0] - exact)) / np.max(np.abs(exact)))
    assert all(errs[i + 1] < 0.5 * errs[i] for i in range(4)), errs


def test_g4_matches_its_closed_form():
    # order 4 in 3D: G4 = G2 + exp(-rho^2/2) / (2 (2 pi)^{3/2} sigma), rho = r / sigma
    sig = 0.3
    r = np.array([0.0, 0.05, 0.3, 0.9, 2.0])
    ref = green.g2_3d(r, sig) + np.exp(-(r / sig) ** 2 / 2) / (2 * (2 * math.pi) ** 1.5 * sig)
    np.testing.assert_allclose(green.green(3, r, sig, "G4"), ref, rtol=1e-14)


# ---------------------------------------------------------------------------
# spectral (sharp cut-off) kernel, 3D
# ---------------------------------------------------------------------------
def test_spectral_kernel_laplacian_is_the_band_limited_delta():
    # -lap [Si(kc r)/(2 pi^2 r)] = (sin(kc r) - kc r cos(kc r)) / (2 pi^2 r^3), the inverse
    # transform of the indicator of |k| <= kc
    kc = 5.0
    for r in (0.1, 0.5, 1.3, 3.0):
        d = 1e-4
        g = lambda x: float(green.green(3, np.array(x), 0.0, "SPECT", kc))
        g0, gp, gm = g(r), g(r + d), g(r - d)
        lap = (gp - 2 * g0 + gm) / d ** 2 + 2 / r * (gp - gm) / (2 * d)
        zeta = (math.sin(kc * r) - kc * r * math.cos(kc * r)) / (2 * math.pi ** 2 * r ** 3)
        assert abs(-lap - zeta) < 1e-6 * kc ** 3
    # r -> 0 limit
    assert abs(float(green.green(3, np.array(1e-9), 0.0, "SPECT", kc)) - kc / (2 * math.pi ** 2)) < 1e-12


def test_spectral_kernel_beats_g2_on_a_resolved_blob():
    from scipy import special
    n = 32
    h = 1.0 / n
    x = -0.5 + h * (np.arange(n) + 0.5)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    R = np.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    s = 0.08
    om = np.exp(-R ** 2 / (2 * s * s)) / (2 * math.pi * s * s) ** 1.5
    exact = special.erf(R / (math.sqrt(2) * s)) / (4 * math.pi * R)
    errs = {}
    for kern in ("G2", "SPECT"):
        d = Desc(3, (n,) * 3, (-0.5,) * 3, (0.5,) * 3, ("U",) * 3, True, rhs_scale=-1.0, sigma=2 * h, kernel=kern)
        psi, _ = oracle.solve(d, om[None])
        errs[kern] = np.max(np.abs(psi[0] - exact)) / np.max(np.abs(exact))
    assert errs["SPECT"] < 0.1 * errs["G2"], errs


# ---------------------------------------------------------------------------
# regular grids (N_c + 1 nodes per axis, padded to the smallest 2^p or 3*2^p >= 2 N_c + 1)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dim,n", [(3, 6), (3, 7), (2, 12), (2, 10)])
def test_direct_sum_regular_grid(dim, n):
    # the aperiodic sum over the N_c + 1 nodes of a regular grid, written out directly
    rng = np.random.default_rng(n + 7 * dim)
    d = Desc(dim, (n, n + 2, n)[:dim], (-0.5,) * dim, (0.5, 0.7, 0.4)[:dim], ("U",) * dim, False,
             rhs_scale=-1.3, sigma=0.09)
    f = rng.normal(size=d.shape())
    psi, _ = oracle.solve(d, f)
    h = [d.h(a) for a in range(dim)]
    nodes = tuple(d.nodes(a) for a in reversed(range(dim)))
    pts = np.argwhere(np.ones(nodes, dtype=bool))
    ref = np.zeros(len(pts))
    for i, p in enumerate(pts):
        r2 = 0.0
        for k in range(dim):
            r2 = r2 + ((p[k] - pts[:, k]) * h[dim - 1 - k]) ** 2
        ref[i] = 1.3 * np.prod(h) * np.sum(green.green(dim, np.sqrt(r2), 0.09) * f.reshape(-1))
    assert np.max(np.abs(psi[0].reshape(-1) - ref)) < 1e-12 * np.max(np.abs(ref))


def test_padded_length_rule():
    from oracle import unbounded
    for n, M in ((6, 16), (7, 16), (8, 24), (12, 32), (16, 48), (127, 256), (128, 384), (255, 512), (256, 768)):
        d = Desc(1, (n,), (0.0,), (1.0,), ("U",), False, sigma=0.1)
        assert unbounded.padded_length(d, 0) == M
    d = Desc(1, (12,), (0.0,), (1.0,), ("U",), True, sigma=0.1)
    assert unbounded.padded_length(d, 0) == 24


@pytest.mark.parametrize("op,ncomp,dim", [("CURL", 3, 3), ("GRAD", 1, 2)])
def test_sampled_points_match_full_oracle_regular(op, ncomp, dim):
    from oracle import unbounded
    n = (10, 7, 6)[:dim]
    d = Desc(dim, n, (-0.5,) * dim, (0.5, 0.4, 0.3)[:dim], ("U",) * dim, False, op=op, ncomp=ncomp,
             rhs_scale=-1.0, sigma=0.12)
    rng = np.random.default_rng(19)
    f = rng.normal(size=(ncomp,) + d.shape())
    psi, opo = oracle.solve(d, f)
    pts = [tuple(int(rng.integers(0, d.nodes(a))) for a in range(dim)) for _ in range(6)]
    pts += [tuple(0 for _ in n), tuple(d.nodes(a) - 1 for a in range(dim))]
    ps, os_ = unbounded.sample_points(d, f, pts)
    for i, p in enumerate(pts):
        idx = tuple(reversed(p))
        np.testing.assert_allclose(ps[i], psi[(slice(None),) + idx], rtol=1e-11, atol=1e-13)
        np.testing.assert_allclose(os_[i], opo[(slice(None),) + idx], rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("op,ncomp,staggered", [("CURL", 3, True), ("GRAD", 1, True), ("DIV", 3, True),
                                                ("NONE", 2, True), ("CURL", 3, False), ("GRAD", 1, False)])
def test_sampled_lines_match_full_oracle(op, ncomp, staggered):
    # whole lines along each axis (direct sums across, the doubled grid's circular
    # convolution along) equal the full doubled-domain solve on every point of the line;
    # unequal extents and cell sizes per axis, both grid types (regular: padded 3 * 2^p)
    from oracle import unbounded
    n = (10, 8, 6)
    d = Desc(3, n, (-0.5,) * 3, (0.5, 0.4, 0.3), ("U",) * 3, staggered, op=op, ncomp=ncomp, rhs_scale=-1.0,
             sigma=0.12)
    rng = np.random.default_rng(23)
    f = rng.normal(size=(ncomp,) + d.shape())
    psi, opo = oracle.solve(d, f)
    for axis in range(3):
        P, Q = [a for a in range(3) if a != axis]
        pos = [(0, 0), (d.nodes(P) - 1, d.nodes(Q) - 1), (int(rng.integers(0, d.nodes(P))),
                                                          int(rng.integers(0, d.nodes(Q))))]
        ls, lo = unbounded.sample_lines(d, f, axis, pos)
        for i, (iP, iQ) in enumerate(pos):
            idx = [slice(None)] * 4
            idx[1 + 2 - P] = iP
            idx[1 + 2 - Q] = iQ
            np.testing.assert_allclose(ls[i], psi[tuple(idx)], rtol=1e-11, atol=1e-13)
            if opo is not None:
                np.testing.assert_allclose(lo[i], opo[tuple(idx)], rtol=1e-10, atol=1e-12)


# ---------------------------------------------------------------------------
# spectral (sharp cut-off) kernel, 2D
# ---------------------------------------------------------------------------
def test_spectral_kernel_2d_laplacian_is_the_band_limited_delta():
    # -lap G = kc J1(kc r) / (2 pi r): the inverse 2D transform of the indicator of |k| <= kc
    kc = 5.0
    g = lambda x: float(green.green(2, np.array(x), 0.0, "SPECT", kc))
    for r in (0.1, 0.5, 1.3, 3.0, 7.7):
        d = 1e-4
        g0, gp, gm = g(r), g(r + d), g(r - d)
        lap = (gp - 2 * g0 + gm) / d ** 2 + 1 / r * (gp - gm) / (2 * d)
        zeta = kc * special.j1(kc * r) / (2 * math.pi * r)
        assert abs(-lap - zeta) < 1e-6 * kc ** 2
    # r -> 0 limit and the gauge: G + ln(r) / (2 pi) -> 0 in the far field
    assert abs(g(0.0) - (math.log(kc / 2) + 0.5772156649015329) / (2 * math.pi)) < 1e-15
    for r in (400.0, 2000.0):
        assert abs(g(r) + math.log(r) / (2 * math.pi)) < 2.0 / (kc * r) ** 1.5


def test_spectral_kernel_2d_beats_g2_on_a_resolved_blob():
    # a Gaussian blob of width s: the free-space potential of lap(psi) = -blob is
    # -(ln r + E1(r^2 / (2 s^2)) / 2) / (2 pi) (the 2D G2 closed form with sigma = s)
    n = 64
    h = 1.0 / n
    x = -0.5 + h * (np.arange(n) + 0.5)
    Y, X = np.meshgrid(x, x, indexing="ij")
    R = np.sqrt(X ** 2 + Y ** 2)
    s = 0.06
    om = np.exp(-R ** 2 / (2 * s * s)) / (2 * math.pi * s * s)
    exact = green.g2_2d(R, s)
    errs = {}
    for kern in ("G2", "SPECT"):
        d = Desc(2, (n,) * 2, (-0.5,) * 2, (0.5,) * 2, ("U",) * 2, True, rhs_scale=-1.0, sigma=2 * h, kernel=kern)
        psi, _ = oracle.solve(d, om[None])
        errs[kern] = np.max(np.abs(psi[0] - exact)) / np.max(np.abs(exact))
    assert errs["SPECT"] < 0.1 * errs["G2"], errs


def test_int_one_minus_j0_hypergeometric_form_matches_quadrature():
    # the closed form used by the oracle against direct quadrature of the integrand
    x = np.concatenate([np.linspace(0.0, 50.0, 101), [123.4, 777.7, 2345.6]])
    np.testing.assert_allclose(green.int_one_minus_j0(x), green.int_one_minus_j0_quad(x), rtol=2e-15, atol=1e-20)


def test_int_one_minus_j0_closed_forms():
    # F(x) = int_0^x (1 - J0(t)) / t dt: series x^2/8 - x^4/256 for small x, and
    # F(x) - ln(x/2) - gamma = int_x^inf J0(t)/t dt -> -J1(x)/x + 2 J0(x)/x^2 for large x
    F = lambda v: float(green.int_one_minus_j0(np.array([v]))[0])
    for v in (1e-3, 2e-2):
        assert abs(F(v) - (v * v / 8 - v ** 4 / 256 + v ** 6 / 13824)) < 1e-14 * v * v
    for v in (300.0, 1500.0):
        tail = -special.j1(v) / v + 2 * special.j0(v) / v ** 2
        assert abs(F(v) - math.log(v / 2) - 0.5772156649015329 - tail) < 10.0 / v ** 3
