"""Independent pins for the FP64 oracle.

Each check compares the oracle with something that does not come from the
oracle: a brute-force DFT, a closed-form Fourier transform, an exact
invariant, or a numerical Hankel transform.  Every check takes the oracle
module as an argument so that ``test_oracle_mutants.py`` can run the same
checks against deliberately broken copies of it.  A check raises
AssertionError on failure.
"""
from __future__ import annotations

import math

import numpy as np

from paper_1709_06999_gb300 import synth

ARCSEC = synth.ARCSEC


# ----------------------------------------------------------------------------
# brute-force references (written from the visibility definition, Sect. 3.1:
# V(u, v) = sum over pixels of I(x, y) exp(+2 pi i (u x + v y)); the sign is
# App. D's, see the phase-convention reading)
# ----------------------------------------------------------------------------

def pixel_xy(nxy, dxy):
    k = np.arange(nxy, dtype=np.float64)
    return (nxy // 2 - k) * dxy, (nxy // 2 - k) * dxy


def direct_dft(img, dxy, u, v):
    """O(N^2) per point: V(u_k, v_k) = sum_ij img_ij exp(+2 pi i (u x_j + v y_i))."""
    n = img.shape[0]
    x, y = pixel_xy(n, dxy)
    u = np.atleast_1d(u)
    v = np.atleast_1d(v)
    ex = np.exp(2j * np.pi * np.outer(u, x))        # (K, N) over columns j
    ey = np.exp(2j * np.pi * np.outer(v, y))        # (K, N) over rows i
    return np.einsum("ki,ij,kj->k", ey, img, ex)


def node_uv(nxy, dxy, both_signs=True, drop_edges=True):
    """uv coordinates of grid nodes (u = c du, v = (r - N/2) du)."""
    du = 1.0 / (nxy * dxy)
    h = nxy // 2
    cs = np.arange(-(h - 1) if both_signs else 0, h)
    rs = np.arange(-(h - 1), h) if drop_edges else np.arange(-h, h)
    U, Vv = np.meshgrid(cs * du, rs * du)
    return U.ravel(), Vv.ravel()


def normwise(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


# ----------------------------------------------------------------------------
# checks
# ----------------------------------------------------------------------------

def check_half_spectrum_bruteforce(O, sizes=(4, 8, 16, 32), seed=11):
    """Every node of the half spectrum equals the direct DFT at that (u, v)."""
    rng = np.random.default_rng(seed)
    for n in sizes:
        dxy = 1.3e-7
        img = rng.standard_normal((n, n))
        G = O.half_spectrum(img)
        du = 1.0 / (n * dxy)
        r, c = np.meshgrid(np.arange(n), np.arange(n // 2 + 1), indexing="ij")
        ref = direct_dft(img, dxy, (c * du).ravel(), ((r - n // 2) * du).ravel()).reshape(r.shape)
        err = np.max(np.abs(G - ref)) / np.max(np.abs(ref))
        assert err < 1e-13, (n, err)


def check_sample_nodes_bruteforce(O, sizes=(4, 8, 16, 32), seed=12):
    """sample_image at nodes of both half planes (u < 0 through the Hermitian
    fold) equals the direct DFT, with PA = 0 and no offset."""
    rng = np.random.default_rng(seed)
    for n in sizes:
        dxy = 2.1e-7
        img = rng.standard_normal((n, n))
        u, v = node_uv(n, dxy)
        V = O.sample_image(img, dxy, u, v)
        ref = direct_dft(img, dxy, u, v)
        assert normwise(V, ref) < 1e-13, n


def check_point_source_nodes(O):
    """A single pixel of flux F at (i, j) has V = F exp(+2 pi i (u x_j + v y_i))."""
    n, dxy, F = 16, 1e-7, 0.7
    for (i, j) in [(3, 11), (12, 5), (8, 8), (0, 1)]:
        img = np.zeros((n, n))
        img[i, j] = F
        x, y = pixel_xy(n, dxy)
        u, v = node_uv(n, dxy)
        V = O.sample_image(img, dxy, u, v)
        ref = F * np.exp(2j * np.pi * (u * x[j] + v * y[i]))
        assert np.max(np.abs(V - ref)) < 1e-13 * F, (i, j)


def check_centred_point_any_geometry(O, seed=13):
    """A centred point source has a constant spectrum, which bilinear
    interpolation reproduces exactly, so for any PA and offset
    V = F exp(+2 pi i (u dRA + v dDec)) at every uv point (Sect. 3.2)."""
    rng = np.random.default_rng(seed)
    n, dxy, F = 64, 0.02 * ARCSEC, 1.3
    img = np.zeros((n, n))
    img[n // 2, n // 2] = F
    u, v = synth.uv_loguniform(500, 1e3, 0.4 / dxy, rng)
    for PA, dRA, dDec in [(0.0, 0.3 * ARCSEC, -0.1 * ARCSEC), (0.7, -0.2 * ARCSEC, 0.45 * ARCSEC),
                          (2.9, 0.05 * ARCSEC, 0.0)]:
        V = O.sample_image(img, dxy, u, v, dRA=dRA, dDec=dDec, PA=PA)
        ref = F * np.exp(2j * np.pi * (u * dRA + v * dDec))
        assert np.max(np.abs(V - ref)) < 1e-12 * F, PA


def check_shift_equals_phase(O):
    """Moving a point source by whole pixels in the image equals the phase
    factor of the same offset applied to the centred source (Sect. 3.2),
    at the grid nodes where both are exact."""
    n, dxy = 32, 0.05 * ARCSEC
    x, y = pixel_xy(n, dxy)
    u, v = node_uv(n, dxy)
    centred = np.zeros((n, n))
    centred[n // 2, n // 2] = 1.0
    for (i, j) in [(10, 20), (25, 4)]:
        moved = np.zeros((n, n))
        moved[i, j] = 1.0
        a = O.sample_image(moved, dxy, u, v)
        b = O.sample_image(centred, dxy, u, v, dRA=x[j], dDec=y[i])
        assert np.max(np.abs(a - b)) < 1e-12, (i, j)


def check_multi_source_equals_composite_image(O):
    """K copies placed in the image by whole pixels, with amplitudes, have at
    the grid nodes exactly the visibilities of the centred model times the
    amplitude-weighted sum of the copies' phase factors (Sect. 3.1, 3.2)."""
    n, dxy = 32, 0.05 * ARCSEC
    x, y = pixel_xy(n, dxy)
    u, v = node_uv(n, dxy)
    base = np.zeros((n, n))
    base[n // 2, n // 2] = 1.0
    base[n // 2 + 1, n // 2 - 2] = 0.5            # an extended, asymmetric model
    spots = [(10, 20, 1.0), (25, 4, -0.7), (3, 30, 2.5)]
    composite = np.zeros((n, n))
    for i, j, a in spots:
        composite += a * np.roll(base, (i - n // 2, j - n // 2), axis=(0, 1))
    want = O.sample_image(composite, dxy, u, v)
    got = O.sample_image_multi(base, dxy, u, v, [x[j] for _, j, _ in spots],
                               [y[i] for i, _, _ in spots], [a for _, _, a in spots])
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))


def check_zero_spacing_total_flux(O, seed=14):
    """V(0, 0) is the sum of the image (Jy/pixel summed is Jy)."""
    rng = np.random.default_rng(seed)
    img = rng.uniform(0, 1, (64, 64))
    V = O.sample_image(img, 1e-7, np.array([0.0]), np.array([0.0]), dRA=1e-6, dDec=-2e-6, PA=0.4)
    assert abs(V[0] - img.sum()) < 1e-13 * img.sum()


def check_hermitian_bitwise(O, seed=15):
    """For a real image V(-u, -v) = conj(V(u, v)); the fold and the phase are
    both conjugate-symmetric, so the equality holds bit for bit."""
    rng = np.random.default_rng(seed)
    n, dxy = 64, 0.03 * ARCSEC
    img = rng.standard_normal((n, n))
    u, v = synth.uv_loguniform(400, 1e3, 0.45 / dxy, rng)
    a = O.sample_image(img, dxy, u, v, dRA=0.07 * ARCSEC, dDec=-0.11 * ARCSEC, PA=1.1)
    b = O.sample_image(img, dxy, -u, -v, dRA=0.07 * ARCSEC, dDec=-0.11 * ARCSEC, PA=1.1)
    assert np.array_equal(a, np.conj(b))


def check_chi2_invariants(O, seed=16):
    """chi2 = 0 when the observation equals the model; chi2 = sum w |n|^2 when
    observation = model + n (Eq. chap6.eq:def.chi.square)."""
    p = synth.small_image_problem(nxy=64, M=2000, seed=seed)
    V = O.sample_image(p.image, p.dxy, p.u, p.v, p.dRA, p.dDec, p.PA)
    assert O.chi2_image(p.image, p.dxy, p.u, p.v, V.real, V.imag, p.w, p.dRA, p.dDec, p.PA) == 0.0
    re, im = V.real + p.noise_re, V.imag + p.noise_im
    got = O.chi2_image(p.image, p.dxy, p.u, p.v, re, im, p.w, p.dRA, p.dDec, p.PA)
    ref = math.fsum((p.w * (p.noise_re ** 2 + p.noise_im ** 2)).tolist())
    assert abs(got - ref) < 1e-12 * ref
    # each term carries its own weight and both parts: a single perturbed point
    # changes chi2 by exactly w_k (dre^2 + dim^2)
    k = 7
    re2, im2 = V.real.copy(), V.imag.copy()
    re2[k] += 0.5
    im2[k] -= 0.25
    got = O.chi2_image(p.image, p.dxy, p.u, p.v, re2, im2, p.w, p.dRA, p.dDec, p.PA)
    assert abs(got - p.w[k] * (0.25 + 0.0625)) < 1e-12


def gaussian_ft(u, v, flux, s_maj, s_min, pa, x0, y0):
    """Closed-form transform of synth.gaussian_image with kernel exp(+2 pi i (u x + v y))."""
    sp, cp = math.sin(pa), math.cos(pa)
    ua = u * sp + v * cp
    ub = u * cp - v * sp
    return flux * np.exp(-2 * math.pi ** 2 * ((s_maj * ua) ** 2 + (s_min * ub) ** 2)) \
        * np.exp(2j * math.pi * (u * x0 + v * y0))


def check_elliptical_gaussian_nodes(O):
    """An elliptical Gaussian (sigma >= 6 px, so aliasing ~exp(-2 pi^2 36) and
    edge truncation are far below rounding) matches its analytic transform at
    the nodes to 1e-10 of the peak."""
    n, dxy = 256, 0.01 * ARCSEC
    args = (1.0, 0.1 * ARCSEC, 0.06 * ARCSEC, 30 * synth.DEG, 0.13 * ARCSEC, -0.21 * ARCSEC)
    img = synth.gaussian_image(n, dxy, *args)
    u, v = node_uv(n, dxy)
    V = O.sample_image(img, dxy, u, v)
    assert normwise(V, gaussian_ft(u, v, *args)) < 1e-10


def check_elliptical_gaussian_between_nodes(O, seed=17):
    """Between nodes the error is the bilinear interpolation error, bounded by
    (du^2/8) (max|V_uu| + max|V_vv|) over the cell; the second derivatives are
    estimated from the analytic transform on a sub-grid of each cell."""
    rng = np.random.default_rng(seed)
    n, dxy = 256, 0.01 * ARCSEC
    args = (1.0, 0.1 * ARCSEC, 0.06 * ARCSEC, 30 * synth.DEG, 0.13 * ARCSEC, -0.21 * ARCSEC)
    img = synth.gaussian_image(n, dxy, *args)
    du = 1.0 / (n * dxy)
    u, v = synth.uv_loguniform(300, 1e4, 0.3 / dxy, rng)
    V = O.sample_image(img, dxy, u, v)
    ref = gaussian_ft(u, v, *args)
    # Hermitian partner for u < 0 lives in the u >= 0 grid
    uf = np.where(u < 0, -u, u)
    vf = np.where(u < 0, -v, v)
    c0 = np.floor(uf / du)
    r0 = np.floor(vf / du)
    t = np.linspace(0, 1, 9)
    h = du / 8
    bound = np.zeros(u.size)
    for a in t:
        for b in t:
            uu = (c0 + a) * du
            vv = (r0 + b) * du
            f = lambda du_, dv_: gaussian_ft(uu + du_, vv + dv_, *args)  # noqa: E731
            fuu = np.abs((f(h, 0) - 2 * f(0, 0) + f(-h, 0)) / h ** 2)
            fvv = np.abs((f(0, h) - 2 * f(0, 0) + f(0, -h)) / h ** 2)
            bound = np.maximum(bound, fuu + fvv)
    bound = bound * du ** 2 / 8 * 1.05 + 1e-13
    err = np.abs(V - ref)
    assert np.all(err <= bound), float(np.max(err / bound))
    # and the bound is not vacuous: the interpolation error is visible
    assert np.max(err) > 1e-6


def check_sweep_gaussian_hankel(O):
    """sweep + transform of I(r) = exp(-r^2/a^2) matches the closed-form Hankel
    transform (Eq. eq:visibility.analytic): V(rho) = pi a^2 exp(-pi^2 a^2 rho^2);
    inclined by inc, V(u, v) = cos(inc) V_face(sqrt(u^2 cos^2 inc + v^2))."""
    n, dxy = 256, 0.01 * ARCSEC
    a = 20 * dxy
    for inc in (0.0, 60 * synth.DEG):
        rmax = (n / 2) * math.sqrt(2) * dxy / math.cos(inc) * 1.01
        dR = a / 2000
        nr = int(rmax / dR) + 2
        r = dR * np.arange(nr)
        I = np.exp(-(r / a) ** 2)
        u, v = node_uv(n, dxy)
        V = O.sample_profile(I, 0.0, dR, n, dxy, u, v, inc=inc)
        rho = np.sqrt((u * math.cos(inc)) ** 2 + v ** 2)
        ref = math.cos(inc) * math.pi * a * a * np.exp(-(math.pi * a * rho) ** 2)
        assert normwise(V, ref) < 1e-6, inc


def paper_templates():
    """Brightness templates (a), (b), (d) of Sect. 5 (profiles in Jy/sr, r in radians)."""
    A = ARCSEC
    g = lambda r, c, w: np.exp(-(((r - c) / w) ** 2))  # noqa: E731
    return {
        "a": lambda r: g(r, 0.0, 0.2 * A) + 0.3 * g(r, 0.4 * A, 0.15 * A),
        "b": lambda r: g(r, 0.5 * A, 0.1 * A),
        "d": lambda r: g(r, 0.2 * A, 0.1 * A) + 0.7 * g(r, 0.5 * A, 0.05 * A) + 0.2 * g(r, 0.7 * A, 0.03 * A),
    }


def hankel_quad(prof, rho, rmax):
    """Numerical V(rho) = 2 pi int_0^rmax I(r) J0(2 pi rho r) r dr (Eq. eq:visibility.analytic)."""
    from scipy.integrate import quad
    from scipy.special import j0
    out = np.empty(rho.size)
    for k, p in enumerate(rho):
        val, _ = quad(lambda r: prof(r) * j0(2 * math.pi * p * r) * r, 0.0, rmax, limit=400,
                      epsabs=0.0, epsrel=1e-10)
        out[k] = 2 * math.pi * val
    return out


def check_paper_templates_hankel(O, keys=("a", "b", "d")):
    """sample_profile of the smooth templates of Sect. 5 matches the numerical
    Hankel transform at grid nodes with baselines 10-1000 klambda; the paper
    finds fractional differences below 1e-5, which is the bound used here
    (normwise, at nodes, where no interpolation error enters)."""
    n, dxy = 512, 0.005 * ARCSEC
    du = 1.0 / (n * dxy)
    dR = dxy / 50
    rmax = (n / 2) * math.sqrt(2) * dxy * 1.01
    nr = int(rmax / dR) + 2
    r = dR * np.arange(nr)
    cs = np.arange(0, 14)
    rs = np.arange(-13, 14)
    U, Vv = np.meshgrid(cs * du, rs * du)
    u, v = U.ravel(), Vv.ravel()
    rho = np.hypot(u, v)
    keep = (rho >= 1e4) & (rho <= 1e6)
    u, v, rho = u[keep], v[keep], rho[keep]
    for key in keys:
        prof = paper_templates()[key]
        V = O.sample_profile(prof(r), 0.0, dR, n, dxy, u, v)
        ref = hankel_quad(prof, rho, 2.5 * ARCSEC)
        assert normwise(V, ref) < 1e-5, key
        assert np.max(np.abs(V.imag)) < 1e-12 * np.max(np.abs(V.real)), key


def check_bilinear_reproduces_bilinear(O, seed=18):
    """bilinear() reproduces any function a + b iv + c iu + d iv iu exactly,
    and evaluates arguments beyond the node range at the nearest edge."""
    rng = np.random.default_rng(seed)
    nrow, ncol = 9, 6
    a, b, c, d = rng.standard_normal(4) + 1j * rng.standard_normal(4)
    R, C = np.meshgrid(np.arange(nrow), np.arange(ncol), indexing="ij")
    grid = a + b * R + c * C + d * R * C
    iv = rng.uniform(0, nrow - 1, 200)
    iu = rng.uniform(0, ncol - 1, 200)
    got = O.bilinear(grid, iv, iu)
    assert np.max(np.abs(got - (a + b * iv + c * iu + d * iv * iu))) < 1e-12
    # exact nodes, including the last row/column
    got = O.bilinear(grid, np.array([0.0, nrow - 1.0, 3.0]), np.array([ncol - 1.0, 0.0, 2.0]))
    assert np.allclose(got, [grid[0, ncol - 1], grid[nrow - 1, 0], grid[3, 2]], rtol=0, atol=1e-13)
    # clamping to the node range
    got = O.bilinear(grid, np.array([-3.0, nrow + 4.0]), np.array([ncol + 0.5, -1.0]))
    assert np.allclose(got, [grid[0, ncol - 1], grid[nrow - 1, 0]], rtol=0, atol=1e-13)


def check_pa_quarter_turn(O):
    """PA rotates the model East of North (Fig. 2): with PA = 90 deg a source
    at (x0, y0) appears at (y0, -x0).  A quarter turn maps nodes to nodes, so
    the check is exact: the rotated sample equals the point-source transform
    of the moved source and the sample of the index-rotated image."""
    n, dxy = 16, 1e-7
    x, y = pixel_xy(n, dxy)
    i0, j0 = 5, 3
    img = np.zeros((n, n))
    img[i0, j0] = 1.0
    u, v = node_uv(n, dxy)
    got = O.sample_image(img, dxy, u, v, PA=math.pi / 2)
    ref = np.exp(2j * np.pi * (u * y[i0] + v * (-x[j0])))
    assert np.max(np.abs(got - ref)) < 1e-12
    moved = np.zeros((n, n))
    moved[n - j0, i0] = 1.0          # pixel of (y0, -x0)
    assert np.max(np.abs(got - O.sample_image(moved, dxy, u, v))) < 1e-12


def check_linearity(O, seed=19):
    rng = np.random.default_rng(seed)
    n, dxy = 32, 0.05 * ARCSEC
    A = rng.standard_normal((n, n))
    B = rng.standard_normal((n, n))
    u, v = synth.uv_loguniform(200, 1e3, 0.4 / dxy, rng)
    kw = dict(dRA=0.1 * ARCSEC, dDec=0.2 * ARCSEC, PA=0.3)
    lhs = O.sample_image(2.0 * A - 0.5 * B, dxy, u, v, **kw)
    rhs = 2.0 * O.sample_image(A, dxy, u, v, **kw) - 0.5 * O.sample_image(B, dxy, u, v, **kw)
    assert normwise(lhs, rhs) < 1e-13


def check_sweep_pixels(O):
    """sweep: Jy/sr -> Jy/px scaling, zero outside [Rmin, Rmax], linear in r,
    centre pixel extrapolated to r = 0, E-W stretch by 1/cos(inc), input kept."""
    n, dxy = 16, 1.0
    Rmin, dR = 1.5, 0.5
    I = 2.0 + 0.25 * np.arange(8)           # linear in r: I(r) = 2 + 0.5 (r - Rmin)
    keep = I.copy()
    img = O.sweep(I, Rmin, dR, n, dxy, inc=0.0)
    assert np.array_equal(I, keep)
    Rmax = Rmin + dR * 7
    x, y = pixel_xy(n, dxy)
    r = np.hypot(x[None, :], y[:, None])
    inside = (r >= Rmin) & (r <= Rmax)
    ref = np.where(inside, 2.0 + 0.5 * (r - Rmin), 0.0) * dxy * dxy
    ref[n // 2, n // 2] = (2.0 - 0.5 * Rmin) * dxy * dxy
    assert np.max(np.abs(img - ref)) < 1e-13
    # inclination: the pixel at x = 6 dxy, y = 0 sits at r = 6 dxy / cos(inc),
    # the pixel at x = 0, y = 6 dxy at r = 6 dxy
    inc = math.acos(0.8)
    img = O.sweep(I, Rmin, dR, n, 0.3, inc=inc)
    r_exp = 6 * 0.3 / 0.8
    assert abs(img[n // 2, n // 2 - 6] - (2.0 + 0.5 * (r_exp - Rmin)) * 0.09) < 1e-13
    assert abs(img[n // 2 - 6, n // 2] - (2.0 + 0.5 * (1.8 - Rmin)) * 0.09) < 1e-13


def check_image_size_table(O):
    """get_image_size against the paper's matrix-size table (Sect. 3.3):
    N_lm of criteria (iia) and (iib) and the pixel size, for 14 ALMA and VLA
    configurations (tests/golden/matrix_sizes.txt)."""
    import os
    arcsec = math.pi / 648000.0
    lam = {"ALMA": 1.3e-3, "VLA": 7.0e-3}
    dish = {"ALMA": 12.0, "VLA": 25.0}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "matrix_sizes.txt")
    with open(path) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 14
    for a, _, bmin, bmax, n1, n2, dth, _ in rows:
        r = np.array([float(bmin), float(bmax)]) / lam[a]
        u, v = r * np.cos([0.3, 2.0]), r * np.sin([0.3, 2.0])
        n, dxy = O.image_size(u, v)
        assert n == int(n1) and abs(dxy / arcsec - float(dth)) <= 0.0005 + 1e-9
        n, _ = O.image_size(u, v, PB=1.5 * lam[a] / dish[a])
        assert n == int(n2)


def check_uv_from_frequency(O):
    """Metres to wavelengths: a 1 km baseline at c / 1 mm = 299.792458 GHz is
    exactly 1e6 wavelengths; 15 m at 100 GHz is 5003.461 wavelengths; the
    conversion is linear in both factors."""
    u, v = O.uv_from_frequency([1000.0, 15.0], [-500.0, 0.0], [299792458000.0, 100e9])
    assert u[0] == 1e6 and v[0] == -5e5
    assert abs(u[1] - 15.0 * 100e9 / 299792458.0) < 1e-9 and v[1] == 0.0
    assert abs(u[1] - 5003.461) < 1e-3



# ----------------------------------------------------------------------------
# full-plane (complex-to-complex) spectrum and the primary beam
# ----------------------------------------------------------------------------

def check_full_spectrum_bruteforce(O, sizes=(4, 8, 16, 32), seed=31):
    """Every node of the full-plane spectrum (both signs of u, no fold) equals
    the direct DFT at u = (c - N/2) du, v = (r - N/2) du."""
    rng = np.random.default_rng(seed)
    for n in sizes:
        dxy = 1.7e-7
        img = rng.standard_normal((n, n))
        G = O.full_spectrum(img)
        du = 1.0 / (n * dxy)
        r, c = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        ref = direct_dft(img, dxy, ((c - n // 2) * du).ravel(),
                         ((r - n // 2) * du).ravel()).reshape(r.shape)
        err = np.max(np.abs(G - ref)) / np.max(np.abs(ref))
        assert err < 1e-13, (n, err)


def check_full_plane_nodes_bruteforce(O, sizes=(8, 16, 32), seed=32):
    """Full-plane sampling at the nodes of both half planes, including the
    u = -N/2 column that only the full plane holds, equals the direct DFT."""
    rng = np.random.default_rng(seed)
    for n in sizes:
        dxy = 2.3e-7
        img = rng.standard_normal((n, n))
        du = 1.0 / (n * dxy)
        u, v = node_uv(n, dxy)
        u = np.concatenate([u, np.full(n - 1, -(n // 2) * du)])
        v = np.concatenate([v, (np.arange(n - 1) - (n // 2 - 1)) * du])
        V = O.sample_image(img, dxy, u, v, full_plane=True)
        assert normwise(V, direct_dft(img, dxy, u, v)) < 1e-13, n


def check_full_plane_matches_half_plane(O, seed=33):
    """Off the nodes, with rotation and offsets, the full-plane and the folded
    half-plane samplings agree to rounding: bilinear interpolation commutes
    with the mirror (u, v) -> (-u, -v) and the spectrum of a real image is
    Hermitian (the paper's C2C versus R2C consistency check)."""
    rng = np.random.default_rng(seed)
    n, dxy = 64, 0.02 * ARCSEC
    img = rng.standard_normal((n, n))
    u, v = synth.uv_loguniform(400, 1e3, 0.4 / dxy, rng)
    for PA, dRA, dDec in [(0.0, 0.0, 0.0), (1.1, 0.2 * ARCSEC, -0.35 * ARCSEC)]:
        a = O.sample_image(img, dxy, u, v, dRA, dDec, PA)
        b = O.sample_image(img, dxy, u, v, dRA, dDec, PA, full_plane=True)
        assert normwise(b, a) < 1e-13, PA


def rotate_to_nodes(ku, kv, du, PA):
    """uv points whose rotated coordinates (Sect. 3.2 equations) are the
    nodes (ku du, kv du): u = R^T k."""
    c, s = math.cos(PA), math.sin(PA)
    return (c * ku + s * kv) * du, (-s * ku + c * kv) * du


def gaussian_beam_ft(u, v, A0, sigma, inc, fwhm, dRA, dDec, PA):
    """Closed-form visibility of a model G(p) = A0 exp(-((x / cos inc)^2 + y^2)
    / (2 sigma^2)) (model coordinates p = (x, y)) that is rotated by PA, moved
    by o = (dRA, dDec) and seen through a circular Gaussian beam of FWHM fwhm
    fixed on the pointing centre, A(s) = exp(-4 ln 2 |s|^2 / fwhm^2).

    Derivation, with k = R u the rotated uv point and b = R o: the model point
    p sits on the sky at R^T p + o, so
        V(u) = e^{2 pi i u.o} int G(p) exp(-c |p + b|^2) e^{2 pi i k.p} dp,
    c = 4 ln 2 / fwhm^2.  Per axis, with a the Gaussian's coefficient and
    alpha = a + c, the integrand is exp(-alpha (x - x0)^2 - (a c / alpha) b^2)
    with x0 = -(c / alpha) b, whose transform is
        sqrt(pi / alpha) exp(-(a c / alpha) b^2) exp(-pi^2 k^2 / alpha)
        e^{2 pi i k x0}."""
    c4 = 4.0 * math.log(2.0) / fwhm ** 2
    cp, sp = math.cos(PA), math.sin(PA)
    ku = u * cp - v * sp
    kv = u * sp + v * cp
    bx = dRA * cp - dDec * sp
    by = dRA * sp + dDec * cp
    out = A0 * np.exp(2j * math.pi * (u * dRA + v * dDec))
    for a, k, b in ((1.0 / (2.0 * (sigma * math.cos(inc)) ** 2), ku, bx),
                    (1.0 / (2.0 * sigma ** 2), kv, by)):
        alpha = a + c4
        x0 = -(c4 / alpha) * b
        out = out * math.sqrt(math.pi / alpha) * math.exp(-(a * c4 / alpha) * b * b) \
            * np.exp(-(math.pi ** 2) * k * k / alpha) * np.exp(2j * math.pi * k * x0)
    return out


def check_beam_gaussian_closed_form(O):
    """A circular Gaussian image through the primary beam, moved and rotated,
    matches the closed-form transform at rotated nodes to 1e-10 (sigma = 12
    px and an effective width >= 9 px: truncation and aliasing are far below
    rounding).  Both the full-plane and the half-plane paths are checked."""
    n, dxy = 256, 0.01 * ARCSEC
    sigma, fwhm, A0 = 12 * dxy, 40 * dxy, 2.5e10
    x, y = pixel_xy(n, dxy)
    img = dxy * dxy * A0 * np.exp(-(x[None, :] ** 2 + y[:, None] ** 2) / (2 * sigma ** 2))
    du = 1.0 / (n * dxy)
    K = np.arange(-40, 41, 3, dtype=np.float64)
    ku, kv = (a.ravel() for a in np.meshgrid(K, K))
    for PA, dRA, dDec in [(0.0, 0.0, 0.0), (0.0, 15 * dxy, -10 * dxy),
                          (0.7, 15 * dxy, -10 * dxy), (2.2, -8 * dxy, 21 * dxy)]:
        u, v = rotate_to_nodes(ku, kv, du, PA)
        ref = gaussian_beam_ft(u, v, A0, sigma, 0.0, fwhm, dRA, dDec, PA)
        for full in (False, True):
            V = O.sample_image(img, dxy, u, v, dRA, dDec, PA, pb_fwhm=fwhm, full_plane=full)
            assert normwise(V, ref) < 1e-10, (PA, dRA, full, normwise(V, ref))


def check_beam_inclined_profile_closed_form(O):
    """An inclined Gaussian profile through the beam (evaluated on the sky, not
    on the deprojected disc) matches the closed form at rotated nodes; the
    tolerance is set by the profile's linear interpolation (dR = sigma / 2000)."""
    n, dxy = 256, 0.01 * ARCSEC
    sigma, fwhm, A0 = 12 * dxy, 30 * dxy, 3.0e10
    inc = 60 * synth.DEG
    rmax = (n / 2) * math.sqrt(2) * dxy / math.cos(inc) * 1.01
    dR = sigma / 2000
    r = dR * np.arange(int(rmax / dR) + 2)
    I = A0 * np.exp(-r ** 2 / (2 * sigma ** 2))
    du = 1.0 / (n * dxy)
    K = np.arange(-40, 41, 4, dtype=np.float64)
    ku, kv = (a.ravel() for a in np.meshgrid(K, K))
    for PA, dRA, dDec in [(0.0, 12 * dxy, 0.0), (1.3, -9 * dxy, 14 * dxy)]:
        u, v = rotate_to_nodes(ku, kv, du, PA)
        V = O.sample_profile(I, 0.0, dR, n, dxy, u, v, dRA, dDec, PA, inc, pb_fwhm=fwhm)
        ref = gaussian_beam_ft(u, v, A0, sigma, inc, fwhm, dRA, dDec, PA)
        assert normwise(V, ref) < 1e-6, (PA, normwise(V, ref))


ALL_CHECKS = [
    check_half_spectrum_bruteforce,
    check_sample_nodes_bruteforce,
    check_point_source_nodes,
    check_centred_point_any_geometry,
    check_shift_equals_phase,
    check_zero_spacing_total_flux,
    check_hermitian_bitwise,
    check_chi2_invariants,
    check_elliptical_gaussian_nodes,
    check_elliptical_gaussian_between_nodes,
    check_sweep_gaussian_hankel,
    check_bilinear_reproduces_bilinear,
    check_pa_quarter_turn,
    check_linearity,
    check_sweep_pixels,
    check_image_size_table,
    check_uv_from_frequency,
    check_multi_source_equals_composite_image,
    check_full_spectrum_bruteforce,
    check_full_plane_nodes_bruteforce,
    check_full_plane_matches_half_plane,
    check_beam_gaussian_closed_form,
    check_beam_inclined_profile_closed_form,
]
