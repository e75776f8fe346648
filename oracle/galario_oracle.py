"""Plain FP64 CPU oracle for the synthetic-visibility / chi-square hot path
of GALARIO (Tazzari, Beaujean & Testi, arXiv 1709.06999).

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously correct
restatement of the method that the CUDA library is checked against.  Only the
test-suite, the package smoke check and the benchmark's CPU-baseline leg may
import it; the library itself never calls it, and it shares no code, table or
helper with the CUDA path.

Everything is computed in float64 with numpy.  Two library primitives serve
as steps: ``numpy.fft.rfft2`` (the 2D real-to-complex FFT of Sect. 4) and
``numpy.interp`` (the 1D linear interpolation of the radial profile used in
App. D).  Every other step is written out in the order of App. D:

    sweep (profile -> image)           Sect. 2 "Basic usage", Sect. 4, App. D
    fftshift -> rfft2 -> fftshift(0)   Sect. 4 (shift, FFT, shift), App. D
    rotate (u, v) by PA                Sect. 3.2, rotation equations
    uv -> grid index, Hermitian fold   App. D (indices, negative-u mapping)
    bilinear interpolation             end of Sect. 3.3 (Press et al.)
    translate by (dRA, dDec)           Sect. 3.2 + App. D (phase factor)
    chi-square                         Sect. 3.1, Eq. (chap6.eq:def.chi.square)

Two variants extend that path: the primary-beam factor A (Sect. 2.1, and
assumption (ii) of the first release's list) multiplied into the image before
the transform, and the complex-to-complex full-plane spectrum (whose agreement
with the real-to-complex one the paper names as a consistency check, Sect. 5)
sampled without the Hermitian fold; ``numpy.fft.fft2`` serves as its step.

Readings of points the paper leaves open or states inconsistently are listed
in the design notes; the ones that change arithmetic are repeated in the
docstrings below.  Pins: every function here is checked, on the CPU, against
something other than itself (brute-force DFT, closed-form transforms,
invariants) in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "pixel_coordinates",
    "primary_beam",
    "full_spectrum",
    "sample_full_spectrum",
    "sweep",
    "half_spectrum",
    "rotate_uv",
    "uv_to_index",
    "image_size",
    "uv_from_frequency",
    "sample_image_multi",
    "chi2_image_multi",
    "chi2_profile_multi",
    "bilinear",
    "sample_spectrum",
    "sample_image",
    "sample_profile",
    "chi2",
    "chi2_image",
    "chi2_profile",
    "uv_extent",
]


def pixel_coordinates(nxy: int, dxy: float):
    """Sky offsets of the pixel centres of an nxy x nxy image (radians).

    Column j sits at x_j = (nxy/2 - j) * dxy and row i at y_i = (nxy/2 - i) *
    dxy: East is to the left, North to the top, and the origin (l, m) = (0, 0)
    is the centre pixel (nxy/2, nxy/2).  Sect. 2 (image orientation), Sect.
    3.3 (origin at the image centre), App. D (mesh-grid construction).
    """
    half = nxy // 2
    idx = np.arange(nxy, dtype=np.float64)
    x = (half - idx) * dxy
    y = (half - idx) * dxy
    return x, y


def sweep(intensity, Rmin: float, dR: float, nxy: int, dxy: float, inc: float = 0.0):
    """Image (Jy/pixel) of an axisymmetric profile I(r) (Jy/sr) seen at inclination inc.

    Sect. 2 (sampleProfile: azimuthal sweep of I(r) over 2*pi, inclination
    along the line of sight) and App. D (py_chi2Profile).  Steps:

    1. radial nodes r_n = Rmin + n * dR, n = 0 .. nr-1;
    2. pixel radius r_ij = sqrt((x_j / cos(inc))**2 + y_i**2): the East-West
       axis is stretched by 1/cos(inc), i.e. the disc is tilted about the
       North-South axis (Fig. 2 caption);
    3. 1D *linear* interpolation of I at r_ij, zero outside [r_0, r_{nr-1}]
       (App. D uses interp1d(kind='linear', fill_value=0)); the text's
       "bilinear as in Press" is read as this 1D interpolation;
    4. Jy/sr -> Jy/pixel by multiplying with dxy**2 (App. D);
    5. the centre pixel takes the linear extrapolation of the first two
       profile samples to r = 0 (App. D, f_center).

    The input array is not modified (App. D scales it in place; the library
    must not, and neither does this oracle).
    """
    I = np.asarray(intensity, dtype=np.float64)
    nr = I.shape[0]
    if nr < 2:
        raise ValueError("profile needs at least two samples")
    radii = Rmin + dR * np.arange(nr, dtype=np.float64)
    x, y = pixel_coordinates(nxy, dxy)
    xs = x / math.cos(inc)
    r = np.sqrt(xs[None, :] ** 2 + y[:, None] ** 2)
    img = np.interp(r, radii, I, left=0.0, right=0.0)
    img *= dxy * dxy
    slope = (I[1] - I[0]) / (radii[1] - radii[0])
    centre = I[0] + slope * (0.0 - radii[0])
    img[nxy // 2, nxy // 2] = centre * dxy * dxy
    return img


def half_spectrum(image):
    """Half-plane spectrum G of a real nxy x nxy image, origin-centred on both sides.

    Sect. 4: the image origin is at the centre pixel while the FFT expects it
    at [0, 0], so the image is shifted, transformed real-to-complex and the
    result is shifted back along the v axis (App. D: fftshift, rfft2,
    fftshift over axis 0).  Unnormalised forward transform e^{-2 pi i k n / N}.
    G has nxy rows (v; row nxy/2 is v = 0) and nxy/2 + 1 columns (u >= 0);
    cell (r, c) is the visibility at u = c * du, v = (r - nxy/2) * du with
    du = 1 / (nxy * dxy).
    """
    img = np.asarray(image, dtype=np.float64)
    n0, n1 = img.shape
    if n0 != n1 or n0 % 2:
        raise ValueError("image must be square with an even side")
    centred = np.fft.fftshift(img)
    return np.fft.fftshift(np.fft.rfft2(centred), axes=0)


def rotate_uv(u, v, PA: float):
    """(u', v') = rotation of the uv points used for a model at position angle PA.

    Sect. 3.2: u' = u cos PA - v sin PA, v' = u sin PA + v cos PA (the
    equations are taken literally; the text calls this a rotation by -PA).
    """
    c, s = math.cos(PA), math.sin(PA)
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    return u * c - v * s, u * s + v * c


def rotate_offsets(dRA: float, dDec: float, PA: float):
    """(dRA', dDec') = 2 pi R (dRA, dDec): the offsets rotated with the same
    matrix as the uv points, in radians per wavelength (Sect. 3.2, App. D)."""
    c, s = math.cos(PA), math.sin(PA)
    dRA_rot = 2.0 * math.pi * (dRA * c - dDec * s)
    dDec_rot = 2.0 * math.pi * (dRA * s + dDec * c)
    return dRA_rot, dDec_rot


def phase_factor(urot, vrot, dRA_rot, dDec_rot):
    """exp(+i theta), theta = u' dRA' + v' dDec' (Sect. 3.2; the sign is App. D's)."""
    theta = urot * dRA_rot + vrot * dDec_rot
    return np.cos(theta) + 1j * np.sin(theta)


def uv_to_index(urot, vrot, nxy: int, dxy: float):
    """Fractional grid indices (row iv, column iu) of rotated uv points, and the fold mask.

    App. D: du = 1 / (nxy * dxy); iu = |u'| / du; iv = nxy/2 + v'/du, except
    that points with u' < 0 (strictly) use the Hermitian partner (-u', -v'),
    i.e. iv = nxy/2 - v'/du, and their sampled value is conjugated.
    """
    du = 1.0 / (nxy * dxy)
    neg = urot < 0.0
    iu = np.abs(urot) / du
    iv = nxy / 2.0 + np.where(neg, -vrot, vrot) / du
    return iv, iu, neg


def bilinear(grid, iv, iu):
    """Bilinear interpolation of a node grid at fractional (row, column) positions.

    End of Sect. 3.3 (Press et al.): the value at a point is inferred from the
    four closest grid nodes assuming linear variation along each axis.  App. D
    performs this with a degree-1, zero-smoothing spline on the nodes
    0..nrow-1, 0..ncol-1, which evaluates arguments beyond the node range at
    the range edge; the same clamping is applied here.  The cell is
    (floor(idx), floor(idx) + 1) except at the last node, where the last cell
    is used with fraction 1.
    """
    G = np.asarray(grid)
    nrow, ncol = G.shape
    fv = np.clip(np.asarray(iv, dtype=np.float64), 0.0, nrow - 1.0)
    fu = np.clip(np.asarray(iu, dtype=np.float64), 0.0, ncol - 1.0)
    r0 = np.minimum(np.floor(fv), nrow - 2).astype(np.int64)
    c0 = np.minimum(np.floor(fu), ncol - 2).astype(np.int64)
    tv = fv - r0
    tu = fu - c0
    return ((1.0 - tv) * (1.0 - tu) * G[r0, c0]
            + (1.0 - tv) * tu * G[r0, c0 + 1]
            + tv * (1.0 - tu) * G[r0 + 1, c0]
            + tv * tu * G[r0 + 1, c0 + 1])


def sample_spectrum(G, nxy: int, dxy: float, u, v, dRA: float = 0.0, dDec: float = 0.0,
                    PA: float = 0.0):
    """Visibilities at (u, v) from a half spectrum G: rotate, index, interpolate, translate.

    Sect. 3.2 and App. D.  The offsets are rotated with the same matrix as the
    uv points and the phase factor is exp(+i theta) with
    theta = 2 pi (u' dRA' + v' dDec').  The text writes the factor with a
    minus sign; App. D (and the orientation of its pixel grid) fix the plus
    sign, under which a source moved East by dRA acquires exp(+2 pi i u dRA).
    """
    urot, vrot = rotate_uv(u, v, PA)
    dRA_rot, dDec_rot = rotate_offsets(dRA, dDec, PA)
    iv, iu, neg = uv_to_index(urot, vrot, nxy, dxy)
    vis = bilinear(G, iv, iu)
    vis = np.where(neg, np.conj(vis), vis)
    return vis * phase_factor(urot, vrot, dRA_rot, dDec_rot)


FOUR_LN2 = 4.0 * math.log(2.0)


def primary_beam(nxy: int, dxy: float, fwhm: float, dRA: float = 0.0, dDec: float = 0.0,
                 PA: float = 0.0):
    """Normalised primary-beam response A at the sky position of every model pixel.

    Sect. 2.1: the visibility is the transform of A I, A being the antenna
    pattern normalised to 1 at the pointing centre; its central lobe is close
    to a Gaussian of full width at half maximum K lambda / D.  Reading: A(s) =
    exp(-4 ln 2 |s|^2 / fwhm^2), circular, centred on the phase centre s = 0.

    A model pixel is placed on the sky by the same geometry as its
    visibilities (Sect. 3.2): with (u', v') = R (u, v) (rotate_uv) and the
    phase exp(+2 pi i (u dRA + v dDec)), pixel p = (x_j, y_i) contributes
    exp(+2 pi i u . (R^T p + o)), o = (dRA, dDec), so it sits at
        s_x =  x cos PA + y sin PA + dRA,   s_y = -x sin PA + y cos PA + dDec.
    The beam stays on the pointing centre while the model moves.
    """
    if not (fwhm > 0.0):
        raise ValueError("the beam width must be positive")
    x, y = pixel_coordinates(nxy, dxy)
    X = x[None, :]
    Y = y[:, None]
    c, s = math.cos(PA), math.sin(PA)
    sx = X * c + Y * s + dRA
    sy = -X * s + Y * c + dDec
    return np.exp(-FOUR_LN2 * (sx * sx + sy * sy) / (fwhm * fwhm))


def full_spectrum(image):
    """Full-plane spectrum of a square image by the complex-to-complex 2D FFT.

    The same transform as half_spectrum (shift, forward FFT e^{-2 pi i k n / N},
    shift) but complex-to-complex and shifted back along both axes, so both
    signs of u are kept: cell (r, c) is the visibility at u = (c - nxy/2) du,
    v = (r - nxy/2) du.  The paper checks this transform against the
    real-to-complex one (Sect. 5, consistency checks).
    """
    img = np.asarray(image, dtype=np.complex128)
    n0, n1 = img.shape
    if n0 != n1 or n0 % 2:
        raise ValueError("image must be square with an even side")
    return np.fft.fftshift(np.fft.fft2(np.fft.fftshift(img)))


def sample_full_spectrum(Gf, nxy: int, dxy: float, u, v, dRA: float = 0.0, dDec: float = 0.0,
                         PA: float = 0.0):
    """Visibilities at (u, v) from a full-plane spectrum: rotate, index, interpolate, translate.

    As sample_spectrum, without the Hermitian fold: iu = nxy/2 + u'/du and
    iv = nxy/2 + v'/du on the full node grid (rows and columns 0 .. nxy-1,
    u and v from -nxy/2 to nxy/2 - 1 cells), clamped to it like App. D's
    spline; no conjugation.
    """
    urot, vrot = rotate_uv(u, v, PA)
    dRA_rot, dDec_rot = rotate_offsets(dRA, dDec, PA)
    du = 1.0 / (nxy * dxy)
    iu = nxy / 2.0 + urot / du
    iv = nxy / 2.0 + vrot / du
    vis = bilinear(Gf, iv, iu)
    return vis * phase_factor(urot, vrot, dRA_rot, dDec_rot)


def sample_image(image, dxy: float, u, v, dRA: float = 0.0, dDec: float = 0.0, PA: float = 0.0,
                 pb_fwhm: float = 0.0, full_plane: bool = False):
    """Synthetic visibilities (Jy) of a model image (Jy/pixel) at uv points (wavelengths).

    Sect. 2 (sampleImage) and Fig. 3: shift, FFT, shift, then sampling.
    pb_fwhm > 0 multiplies the image by primary_beam() first (the image is
    then the bare brightness I, not A I); full_plane selects the
    complex-to-complex spectrum and the unfolded sampling.
    """
    img = np.asarray(image, dtype=np.float64)
    n = img.shape[0]
    if pb_fwhm > 0.0:
        img = img * primary_beam(n, dxy, pb_fwhm, dRA, dDec, PA)
    if full_plane:
        return sample_full_spectrum(full_spectrum(img), n, dxy, u, v, dRA, dDec, PA)
    return sample_spectrum(half_spectrum(img), n, dxy, u, v, dRA, dDec, PA)


def sample_profile(intensity, Rmin: float, dR: float, nxy: int, dxy: float, u, v,
                   dRA: float = 0.0, dDec: float = 0.0, PA: float = 0.0, inc: float = 0.0,
                   pb_fwhm: float = 0.0, full_plane: bool = False):
    """Synthetic visibilities of an axisymmetric profile: sweep, then sample_image (Sect. 2, Fig. 3).

    The beam, when given, is evaluated on the sky (pixel positions, not the
    deprojected disc radius)."""
    img = sweep(intensity, Rmin, dR, nxy, dxy, inc)
    return sample_image(img, dxy, u, v, dRA, dDec, PA, pb_fwhm, full_plane)


def chi2(vis, re_obs, im_obs, w):
    """Weighted chi-square of Eq. (chap6.eq:def.chi.square), Sect. 3.1.

    chi2 = sum_k w_k [(Re_obs - Re_mod)^2 + (Im_obs - Im_mod)^2].  The terms are
    formed in float64 and summed with ``math.fsum`` (Shewchuk's exact
    summation), so the sum itself adds no rounding beyond the final one.
    """
    vis = np.asarray(vis)
    dr = np.asarray(re_obs, dtype=np.float64) - vis.real
    di = np.asarray(im_obs, dtype=np.float64) - vis.imag
    terms = np.asarray(w, dtype=np.float64) * (dr * dr + di * di)
    return math.fsum(terms.tolist())


def chi2_image(image, dxy: float, u, v, re_obs, im_obs, w, dRA: float = 0.0, dDec: float = 0.0,
               PA: float = 0.0, pb_fwhm: float = 0.0, full_plane: bool = False):
    """chi2Image of Sect. 2: sample_image followed by the chi-square reduction."""
    vis = sample_image(image, dxy, u, v, dRA, dDec, PA, pb_fwhm, full_plane)
    return chi2(vis, re_obs, im_obs, w)


def chi2_profile(intensity, Rmin: float, dR: float, nxy: int, dxy: float, u, v, re_obs, im_obs, w,
                 dRA: float = 0.0, dDec: float = 0.0, PA: float = 0.0, inc: float = 0.0,
                 pb_fwhm: float = 0.0, full_plane: bool = False):
    """chi2Profile of Sect. 2: sample_profile followed by the chi-square reduction."""
    vis = sample_profile(intensity, Rmin, dR, nxy, dxy, u, v, dRA, dDec, PA, inc, pb_fwhm,
                         full_plane)
    return chi2(vis, re_obs, im_obs, w)


def uv_extent(u, v):
    """Largest baseline length max_k sqrt(u_k^2 + v_k^2) (Sect. 3.3, criterion (i))."""
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    if u.size == 0:
        return 0.0
    return float(np.sqrt(np.max(u * u + v * v)))


# Largest-recoverable-scale constant of criterion (iia); the paper quotes
# Gamma ~ 0.5 in general and 0.6 for ALMA.  Its matrix-size table is
# reproduced with 0.6 only (0.5 gives 512 instead of 1024 for ALMA C43-3).
MRS_GAMMA = 0.6


def image_size(u, v, PB: float = 0.0, f_min: float = 5.0, f_max: float = 2.5):
    """get_image_size of Sect. 3.3: (nxy, dxy) for the uv points.

    Criterion (i): the modelled uv region must reach f_max times the longest
    baseline, nxy * duv / 2 >= f_max * rho_max.  Criterion (iia): the field
    nxy * dxy = 1 / duv must exceed f_min times the largest recoverable scale
    Gamma / rho_min, i.e. duv = rho_min / (Gamma f_min).  Criterion (iib), when
    the primary-beam FWHM PB (radians) is given: the field must also cover the
    beam, duv <= 1 / PB.  nxy is the smallest power of two satisfying (i), and
    dxy = 1 / (nxy duv).

    Readings (the printed equations and the table disagree): the table's
    N_lm (iia) column equals the power of two at or above
    2 f_max Gamma f_min rho_max / rho_min, i.e. criteria (i) and (iia)
    combined -- the printed N_lm equation drops f_max; its N_lm (iib) column
    is reproduced when the field satisfies both (iia) and (iib) (the larger
    of the two image sizes), and its pixel sizes equal 1 / (nxy duv).
    """
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    r = np.sqrt(u * u + v * v)
    r = r[np.isfinite(r)]
    if r.size == 0 or not r.min() > 0.0:
        raise ValueError("need at least one finite, non-zero baseline")
    if not (f_min > 1.0 and f_max > 2.0 and PB >= 0.0):
        raise ValueError("criteria need f_min > 1, f_max > 2, PB >= 0")
    rho_min, rho_max = float(r.min()), float(r.max())
    duv = rho_min / (MRS_GAMMA * f_min)           # (iia)
    if PB > 0.0:
        duv = min(duv, 1.0 / PB)                  # (iib)
    need = 2.0 * f_max * rho_max / duv            # (i)
    mant, expo = math.frexp(need)                 # need = mant * 2**expo, mant in [0.5, 1)
    nxy = 2 ** (expo - 1) if mant == 0.5 else 2 ** expo
    return int(nxy), 1.0 / (nxy * duv)


SPEED_OF_LIGHT = 299792458.0  # m/s, exact by the SI definition of the metre


def uv_from_frequency(u_m, v_m, nu):
    """Baselines in metres observed at frequency nu (Hz) expressed in
    wavelengths, u = u_m nu / c (Sect. 3: uv coordinates are baselines in
    units of the observing wavelength).  With one nu per visibility the
    single-frequency assumption of Sect. 3 is lifted: each visibility samples
    the model at its own uv.  Computed as (u_m nu) / c."""
    u_m = np.asarray(u_m, dtype=np.float64)
    v_m = np.asarray(v_m, dtype=np.float64)
    nu = np.asarray(nu, dtype=np.float64)
    return (u_m * nu) / SPEED_OF_LIGHT, (v_m * nu) / SPEED_OF_LIGHT


def sample_image_multi(image, dxy: float, u, v, dRA, dDec, amp=None, PA: float = 0.0):
    """K copies of one model at different places (end of Sect. 3.1): by
    linearity of the Fourier transform, the sum over k of amp[k] times the
    visibilities of the model displaced by (dRA[k], dDec[k]) (Sect. 3.2), all
    rotated by PA."""
    amp = [1.0] * len(dRA) if amp is None else amp
    total = 0.0
    for a, x, y in zip(amp, dRA, dDec):
        total = total + a * sample_image(image, dxy, u, v, x, y, PA)
    return total


def chi2_image_multi(image, dxy: float, u, v, re_obs, im_obs, w, dRA, dDec, amp=None,
                     PA: float = 0.0):
    """chi-square (Sect. 3.1) of the multi-source model of sample_image_multi."""
    return chi2(sample_image_multi(image, dxy, u, v, dRA, dDec, amp, PA), re_obs, im_obs, w)


def chi2_profile_multi(intensity, Rmin: float, dR: float, nxy: int, dxy: float, u, v, re_obs,
                       im_obs, w, dRA, dDec, amp=None, PA: float = 0.0, inc: float = 0.0):
    """chi-square of K copies of the swept profile (sweep, then sample_image_multi)."""
    img = sweep(intensity, Rmin, dR, nxy, dxy, inc)
    return chi2_image_multi(img, dxy, u, v, re_obs, im_obs, w, dRA, dDec, amp, PA)
