"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input generators only: model images, radial profiles, uv
coverages, weights and noise.  It contains none of the visibility / chi-square
arithmetic; observed visibilities are formed by the caller as "model + noise"
with a model computed elsewhere.  Every generator takes an explicit
``numpy.random.Generator`` or seed, so tests and the benchmark draw identical
inputs.

Units follow the paper (Sect. 2): angles in radians, uv in wavelengths,
images in Jy/pixel, profiles in Jy/sr.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

ARCSEC = math.pi / (180.0 * 3600.0)
DEG = math.pi / 180.0


def _rng(seed):
    return seed if isinstance(seed, np.random.Generator) else np.random.default_rng(seed)


def gaussian_image(nxy: int, dxy: float, flux: float, sigma_major: float, sigma_minor: float,
                   pa: float, x0: float = 0.0, y0: float = 0.0) -> np.ndarray:
    """Elliptical Gaussian of total flux ``flux`` (Jy) sampled at pixel centres (Jy/pixel).

    Pixel (i, j) sits at x = (nxy/2 - j) dxy (East), y = (nxy/2 - i) dxy
    (North).  ``pa`` is the major-axis position angle East of North.
    """
    half = nxy // 2
    idx = np.arange(nxy, dtype=np.float64)
    x = ((half - idx) * dxy)[None, :] - x0
    y = ((half - idx) * dxy)[:, None] - y0
    sp, cp = math.sin(pa), math.cos(pa)
    a = x * sp + y * cp          # along the major axis
    b = x * cp - y * sp          # along the minor axis
    norm = flux * dxy * dxy / (2.0 * math.pi * sigma_major * sigma_minor)
    return norm * np.exp(-0.5 * ((a / sigma_major) ** 2 + (b / sigma_minor) ** 2))


def point_source(nxy: int, flux: float, i: int, j: int) -> np.ndarray:
    img = np.zeros((nxy, nxy))
    img[i, j] = flux
    return img


def exp_disk_image(nxy: int, dxy: float, flux: float, scale: float) -> np.ndarray:
    """Face-on exponential disc exp(-r/scale), normalised to ``flux`` Jy in total."""
    half = nxy // 2
    idx = np.arange(nxy, dtype=np.float64)
    x = ((half - idx) * dxy)[None, :]
    y = ((half - idx) * dxy)[:, None]
    img = np.exp(-np.sqrt(x * x + y * y) / scale)
    return img * (flux / img.sum())


def uv_loguniform(M: int, rho_min: float, rho_max: float, seed) -> tuple[np.ndarray, np.ndarray]:
    """uv points with uniform angle in [0, 2 pi) and log-uniform radius in [rho_min, rho_max]."""
    rng = _rng(seed)
    ang = rng.uniform(0.0, 2.0 * math.pi, M)
    rad = np.exp(rng.uniform(math.log(rho_min), math.log(rho_max), M))
    return rad * np.cos(ang), rad * np.sin(ang)


def weights_uniform(M: int, seed, lo: float = 0.5, hi: float = 2.0) -> np.ndarray:
    return _rng(seed).uniform(lo, hi, M)


def noise(w: np.ndarray, seed) -> tuple[np.ndarray, np.ndarray]:
    """Gaussian noise with sigma = 1/sqrt(w) on Re and Im (Sect. 3.1: w = 1/sigma^2)."""
    rng = _rng(seed)
    sig = 1.0 / np.sqrt(w)
    return rng.standard_normal(w.shape) * sig, rng.standard_normal(w.shape) * sig


def alma_like_uv(M: int, seed, n_ant: int = 43, r_min_m: float = 15.0, r_max_m: float = 3000.0,
                 lat: float = -23.0 * DEG, dec: float = -35.0 * DEG, ha_hours: float = 2.0,
                 n_time: int = 60, freq0_hz: float = 100e9, half_band_hz: float = 3.75e9,
                 metres: bool = False):
    """ALMA-like Earth-rotation tracks, truncated to exactly M points.

    ``n_ant`` antennas at log-uniform radius in [r_min_m, r_max_m] and uniform
    azimuth on a flat site at latitude ``lat``; baselines are projected with
    the standard (X, Y, Z) -> (u, v) transform for hour angles uniformly in
    [-ha, +ha] (n_time steps) and declination ``dec``; channels spread over
    freq0 +- half_band are added until M points exist.  Returns (u, v) in
    wavelengths, or with ``metres`` the baselines in metres and each point's
    frequency in Hz, (u_m, v_m, nu).
    """
    rng = _rng(seed)
    rad = np.exp(rng.uniform(math.log(r_min_m), math.log(r_max_m), n_ant))
    az = rng.uniform(0.0, 2.0 * math.pi, n_ant)
    east, north = rad * np.sin(az), rad * np.cos(az)
    i, j = np.triu_indices(n_ant, 1)
    bE, bN = east[j] - east[i], north[j] - north[i]
    # local (E, N, Up=0) -> equatorial (X, Y, Z)
    X = -math.sin(lat) * bN
    Y = bE
    Z = math.cos(lat) * bN
    H = np.linspace(-ha_hours, ha_hours, n_time) * (math.pi / 12.0)
    sH, cH = np.sin(H)[:, None], np.cos(H)[:, None]
    u_m = (sH * X + cH * Y).ravel()
    v_m = (-math.sin(dec) * cH * X + math.sin(dec) * sH * Y + math.cos(dec) * Z).ravel()
    per_chan = u_m.size
    n_chan = max(1, -(-M // per_chan))
    freqs = freq0_hz + (np.linspace(-half_band_hz, half_band_hz, n_chan) if n_chan > 1 else np.zeros(1))
    if metres:
        um = np.broadcast_to(u_m[None, :], (n_chan, per_chan)).ravel()[:M].copy()
        vm = np.broadcast_to(v_m[None, :], (n_chan, per_chan)).ravel()[:M].copy()
        nu = np.broadcast_to(freqs[:, None], (n_chan, per_chan)).ravel()[:M].copy()
        return um, vm, nu
    c_light = 299792458.0
    scale = freqs / c_light
    u = (u_m[None, :] * scale[:, None]).ravel()[:M]
    v = (v_m[None, :] * scale[:, None]).ravel()[:M]
    return u, v


@dataclass
class ImageProblem:
    """One chi2_image evaluation: image, pixel size, geometry and a uv dataset."""
    image: np.ndarray
    dxy: float
    u: np.ndarray
    v: np.ndarray
    w: np.ndarray
    noise_re: np.ndarray
    noise_im: np.ndarray
    dRA: float
    dDec: float
    PA: float


@dataclass
class ProfileProblem:
    intensity: np.ndarray
    Rmin: float
    dR: float
    nxy: int
    dxy: float
    inc: float
    u: np.ndarray
    v: np.ndarray
    w: np.ndarray
    noise_re: np.ndarray
    noise_im: np.ndarray
    dRA: float
    dDec: float
    PA: float


def small_image_problem(nxy: int = 256, M: int = 10_000, seed: int = 0) -> ImageProblem:
    """Plain FP64 chi2_image case: nxy=256, dxy=0.01", M=1e4.

    Elliptical Gaussian (sigma 0.1"/0.06", PA 30 deg, 1 Jy) plus a 0.5 Jy
    point source at (RA, Dec) = (0.3", -0.2"); uv angle uniform, radius
    log-uniform over [1e4, 0.45/dxy]; w ~ U[0.5, 2]; dRA=0.05", dDec=-0.03",
    PA=0.  Other sizes keep the same recipe with the point source placed at
    the same pixel offset from the centre (clipped into the image).
    """
    dxy = 0.01 * ARCSEC
    rng = np.random.default_rng(seed)
    img = gaussian_image(nxy, dxy, 1.0, 0.1 * ARCSEC, 0.06 * ARCSEC, 30.0 * DEG)
    di, dj = 20, -30                                  # (0.3", -0.2") at 0.01" per pixel
    i = min(max(nxy // 2 + di, 0), nxy - 1)
    j = min(max(nxy // 2 + dj, 0), nxy - 1)
    img[i, j] += 0.5
    u, v = uv_loguniform(M, 1e4, 0.45 / dxy, rng)
    w = weights_uniform(M, rng)
    nre, nim = noise(w, rng)
    return ImageProblem(img, dxy, u, v, w, nre, nim, 0.05 * ARCSEC, -0.03 * ARCSEC, 0.0)


def ring_profile(nr: int, dR: float, Rmin: float, r0: float = 0.5 * ARCSEC,
                 width: float = 0.1 * ARCSEC, power: float = -0.5) -> np.ndarray:
    """Gaussian ring exp(-((r - r0)/width)^2) times (r / 1")^power, in Jy/sr."""
    r = Rmin + dR * np.arange(nr)
    return np.exp(-(((r - r0) / width) ** 2)) * (r / ARCSEC) ** power


def profile_problem(nxy: int = 1024, M: int = 1_000_000, nr: int = 8192, seed: int = 1,
                    dxy: float = 0.005 * ARCSEC) -> ProfileProblem:
    """chi2_profile case: Gaussian ring (r0=0.5", width 0.1") x r^-0.5, nr=8192,
    dR = 4.5"/8192, Rmin = dR/2, inclination 45 deg, nxy=1024, dxy=0.005",
    uv as in the small image case with radius up to 0.45/dxy.

    Other (nxy, dxy, nr) scale the radial extent with the field of view
    (4.5" for a 5.12" field covers the farthest pixel of the 45 deg image)
    and keep the ring at the same place on the sky.
    """
    extent = 4.5 * ARCSEC * (nxy * dxy) / (5.12 * ARCSEC)
    dR = extent / nr
    Rmin = dR / 2
    rng = np.random.default_rng(seed)
    I = ring_profile(nr, dR, Rmin)
    u, v = uv_loguniform(M, 1e4, 0.45 / dxy, rng)
    w = weights_uniform(M, rng)
    nre, nim = noise(w, rng)
    return ProfileProblem(I, Rmin, dR, nxy, dxy, 45.0 * DEG, u, v, w, nre, nim,
                          0.05 * ARCSEC, -0.03 * ARCSEC, 0.0)


def large_image(nxy: int, dxy: float, seed) -> np.ndarray:
    """Three random elliptical Gaussians plus an exp(-r/0.2") disc (1 Jy).

    sigma ~ U[0.02", 0.3"] per axis, centres within +-1", fluxes U[0.1, 1] Jy,
    position angles U[0, pi).
    """
    rng = _rng(seed)
    img = exp_disk_image(nxy, dxy, 1.0, 0.2 * ARCSEC)
    for _ in range(3):
        s1, s2 = sorted(rng.uniform(0.02, 0.3, 2) * ARCSEC, reverse=True)
        img += gaussian_image(nxy, dxy, rng.uniform(0.1, 1.0), s1, s2, rng.uniform(0.0, math.pi),
                              rng.uniform(-1.0, 1.0) * ARCSEC, rng.uniform(-1.0, 1.0) * ARCSEC)
    return img


def large_image_problem(nxy: int = 4096, M: int = 5_000_000, seed: int = 2) -> ImageProblem:
    """Large single-image case: nxy=4096, dxy=0.002", M=5e6 ALMA-like points,
    dRA/dDec ~ U[-0.1", 0.1"], PA ~ U[0, pi)."""
    dxy = 0.002 * ARCSEC
    rng = np.random.default_rng(seed)
    img = large_image(nxy, dxy, rng)
    u, v = alma_like_uv(M, rng)
    w = weights_uniform(M, rng)
    nre, nim = noise(w, rng)
    dRA, dDec = rng.uniform(-0.1, 0.1, 2) * ARCSEC
    PA = rng.uniform(0.0, math.pi)
    return ImageProblem(img, dxy, u, v, w, nre, nim, float(dRA), float(dDec), float(PA))


def keplerian_channel(nxy: int, dxy: float, v_chan: float, r_c: float = 0.8 * ARCSEC,
                      inc: float = 40.0 * DEG, pa: float = 30.0 * DEG, mstar: float = 1.0,
                      dist_pc: float = 140.0, sigma_v: float = 0.25,
                      flux_scale: float = 1.0) -> np.ndarray:
    """One channel map of a Keplerian disc's line emission (Jy/pixel).

    I(r, phi) ~ exp(-r/r_c) exp(-(v_chan - v_K(r) sin(inc) cos(phi))^2 / (2 sigma_v^2)),
    v_K = 29.78 km/s sqrt(mstar / r[au]) with r[au] = r["] * dist_pc; (r, phi)
    are disc-plane polar coordinates of the sky pixel (inclination inc, major
    axis at position angle pa East of North); velocities in km/s.
    """
    c = (np.arange(nxy) - nxy // 2) * dxy
    x = -c[None, :]                     # East to the left, as in the pixel convention
    y = c[:, None]
    cp, sp = math.cos(pa), math.sin(pa)
    xm = x * sp + y * cp                # along the major axis
    ym = (-x * cp + y * sp) / math.cos(inc)
    r = np.sqrt(xm * xm + ym * ym)
    cosphi = np.where(r > 0, xm / np.maximum(r, 1e-30), 0.0)
    r_au = np.maximum(r / ARCSEC * dist_pc, 1e-3)
    vk = 29.78 * np.sqrt(mstar / r_au)
    line = np.exp(-((v_chan - vk * math.sin(inc) * cosphi) ** 2) / (2.0 * sigma_v ** 2))
    img = np.exp(-r / r_c) * line
    total = img.sum()
    return (img * (flux_scale / total if total > 0 else 0.0))


@dataclass
class CubeChannel:
    image: np.ndarray
    dxy: float
    u: np.ndarray
    v: np.ndarray
    w: np.ndarray
    noise_re: np.ndarray
    noise_im: np.ndarray
    dRA: float
    dDec: float
    PA: float


def spectral_cube(n_chan: int = 128, sizes=(512, 1024, 2048), m_lo: int = 100_000,
                  m_hi: int = 2_000_000, fov: float = 5.12 * ARCSEC, seed: int = 3,
                  base_uv=None) -> list[CubeChannel]:
    """Channels of a Keplerian disc cube: per channel a side drawn uniformly
    from ``sizes`` (pixel size fov / side), an observation of M_c ~ U[m_lo, m_hi]
    points subsampled from the ALMA-like layout and scaled by the channel
    frequency (line at 100 GHz, channels 0.5 km/s apart), w ~ U[0.5, 2] and
    noise sigma = 1/sqrt(w).  One set of dRA, dDec, PA for the cube."""
    rng = np.random.default_rng(seed)
    if base_uv is None:
        base_uv = alma_like_uv(m_hi, rng)
    bu, bv = base_uv
    dRA, dDec = (float(a) for a in rng.uniform(-0.1, 0.1, 2) * ARCSEC)
    PA = float(rng.uniform(0.0, math.pi))
    dv = 0.5
    out = []
    for k in range(n_chan):
        nxy = int(sizes[rng.integers(len(sizes))])
        dxy = fov / nxy
        v_chan = (k - (n_chan - 1) / 2) * dv
        scale = 1.0 - v_chan / 299792.458          # frequency of the channel / line frequency
        m = int(rng.integers(m_lo, m_hi + 1))
        sel = rng.choice(bu.size, size=m, replace=False) if m < bu.size else np.arange(bu.size)
        w = weights_uniform(m, rng)
        nre, nim = noise(w, rng)
        out.append(CubeChannel(keplerian_channel(nxy, dxy, v_chan).astype(np.float64), dxy,
                               bu[sel] * scale, bv[sel] * scale, w, nre, nim, dRA, dDec, PA))
    return out


def walker_params(n: int = 64, seed: int = 4) -> list[dict]:
    """Random ring-profile and geometry parameters for MCMC walkers: ring
    radius U[0.3", 0.7"], width U[0.05", 0.15"], power-law exponent U[-1, 0],
    inclination U[0, 70 deg], PA U[0, pi), dRA/dDec U[-0.1", 0.1"]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        out.append(dict(r0=rng.uniform(0.3, 0.7) * ARCSEC, width=rng.uniform(0.05, 0.15) * ARCSEC,
                        power=rng.uniform(-1.0, 0.0), inc=rng.uniform(0.0, 70.0) * DEG,
                        PA=rng.uniform(0.0, math.pi), dRA=rng.uniform(-0.1, 0.1) * ARCSEC,
                        dDec=rng.uniform(-0.1, 0.1) * ARCSEC))
    return out
