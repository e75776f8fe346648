"""Observations registered from baselines in metres with one frequency per
visibility (gal_data_create_freq_*): the library's wavelengths equal
u_m nu / c computed by the oracle, so the chi-square is bitwise that of the
same points registered in wavelengths, and matches the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1709_06999_gb300 import Context, synth

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-6}


@pytest.mark.parametrize("dt", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_metres_and_frequencies(dt):
    ctx = Context(0)
    rng = np.random.default_rng(31)
    M = 150_001   # three channels of the layout, ragged
    u_m, v_m, nu = synth.alma_like_uv(M, rng, metres=True)
    assert len(np.unique(nu)) > 1
    w = synth.weights_uniform(M, rng)
    nre, nim = synth.noise(w, rng)
    nxy, dxy = 512, 0.01 * synth.ARCSEC
    img = synth.large_image(nxy, dxy, rng)
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")  # noqa: E731
    host = lambda t: t.double().cpu().numpy()  # noqa: E731
    tm = [d(a) for a in (u_m, v_m, nu, nre, nim, w)]
    obs_f = ctx.register_freq(*tm)
    # the oracle's wavelengths from the values the device holds, rounded to dt
    u_l, v_l = oracle.uv_from_frequency(host(tm[0]), host(tm[1]), host(tm[2]))
    tl = [d(u_l), d(v_l)] + tm[3:]
    obs_l = ctx.register(*tl)
    image = d(img)
    geo = (0.03 * synth.ARCSEC, -0.02 * synth.ARCSEC, 0.7)
    a = ctx.chi2_image(image, dxy, obs_f, *geo).item()
    b = ctx.chi2_image(image, dxy, obs_l, *geo).item()
    assert a == b
    ref = oracle.chi2_image(host(image), dxy, host(tl[0]), host(tl[1]), host(tl[2]), host(tl[3]),
                            host(tl[4]), *geo)
    assert abs(a - ref) <= TOL[dt] * abs(ref)


def test_single_frequency_reduces_to_the_plain_layout():
    ctx = Context(0)
    rng = np.random.default_rng(32)
    M = 20_000
    u_m, v_m, _ = synth.alma_like_uv(M, rng, metres=True)
    nu = np.full(M, 299792458.0 * 1000.0)        # lambda = 1 mm: u = 1000 u_m
    w = np.ones(M)
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")  # noqa: E731
    obs_f = ctx.register_freq(d(u_m), d(v_m), d(nu), d(w), d(w), d(w))
    obs_l = ctx.register(d(1000.0 * u_m), d(1000.0 * v_m), d(w), d(w), d(w))
    img = d(synth.gaussian_image(256, 0.02 * synth.ARCSEC, 1.0, 0.2 * synth.ARCSEC,
                                 0.1 * synth.ARCSEC, 0.3))
    a = ctx.chi2_image(img, 0.02 * synth.ARCSEC, obs_f, PA=0.4).item()
    b = ctx.chi2_image(img, 0.02 * synth.ARCSEC, obs_l, PA=0.4).item()
    assert abs(a - b) <= 1e-12 * abs(b)     # (u_m nu) / c and 1000 u_m round differently
