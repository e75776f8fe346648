"""Multi-source composition (K offset copies of one model, one FFT) against
the oracle's sum of displaced single-source evaluations."""
import numpy as np
import pytest
import torch

import oracle
from paper_1709_06999_gb300 import Context, GalError, synth

pytestmark = pytest.mark.gpu

TOL_VIS = {torch.float64: 1e-12, torch.float32: 1e-5}
TOL_CHI2 = {torch.float64: 1e-12, torch.float32: 1e-6}
ARC = synth.ARCSEC


def normwise(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def sources(K, seed):
    rng = np.random.default_rng(seed)
    return (list(rng.uniform(-0.4, 0.4, K) * ARC), list(rng.uniform(-0.4, 0.4, K) * ARC),
            list(rng.uniform(0.2, 1.5, K)))


@pytest.mark.parametrize("dt", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("K", [1, 3, 16])
def test_sample_and_chi2_image_multi(dt, K):
    ctx = Context(0)
    p = synth.small_image_problem(nxy=256, M=12_345, seed=40 + K)
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")  # noqa: E731
    h = lambda t: t.double().cpu().numpy()  # noqa: E731
    img, u, v = d(p.image), d(p.u), d(p.v)
    dRA, dDec, amp = sources(K, K)
    PA = 0.6
    got = ctx.sample_image_multi(img, p.dxy, u, v, dRA, dDec, amp, PA).cpu().numpy()
    want = oracle.sample_image_multi(h(img), p.dxy, h(u), h(v), dRA, dDec, amp, PA)
    assert normwise(got[:, 0] + 1j * got[:, 1], want) <= TOL_VIS[dt]
    re, im, w = d(p.noise_re), d(p.noise_im), d(p.w)
    obs = ctx.register(u, v, re, im, w)
    c = ctx.chi2_image_multi(img, p.dxy, obs, dRA, dDec, amp, PA).item()
    ref = oracle.chi2_image_multi(h(img), p.dxy, h(u), h(v), h(re), h(im), h(w), dRA, dDec, amp,
                                  PA)
    assert abs(c - ref) <= TOL_CHI2[dt] * abs(ref)


@pytest.mark.parametrize("dt", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_chi2_profile_multi(dt):
    ctx = Context(0)
    q = synth.profile_problem(nxy=256, M=20_000, nr=512, seed=7, dxy=0.02 * ARC)
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")  # noqa: E731
    h = lambda t: t.double().cpu().numpy()  # noqa: E731
    t = [d(a) for a in (q.u, q.v, q.noise_re, q.noise_im, q.w)]
    obs = ctx.register(*t)
    I = d(q.intensity)
    dRA, dDec, amp = sources(4, 9)
    c = ctx.chi2_profile_multi(I, q.Rmin, q.dR, q.nxy, q.dxy, obs, dRA, dDec, amp, q.inc,
                               0.2).item()
    ref = oracle.chi2_profile_multi(h(I), q.Rmin, q.dR, q.nxy, q.dxy, *[h(x) for x in t], dRA,
                                    dDec, amp, 0.2, q.inc)
    assert abs(c - ref) <= TOL_CHI2[dt] * abs(ref)


@pytest.mark.parametrize("dt", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_one_unit_copy_is_the_single_call(dt):
    ctx = Context(0)
    p = synth.large_image_problem(nxy=1024, M=100_003, seed=5)
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")  # noqa: E731
    img = d(p.image)
    obs = ctx.register(*[d(a) for a in (p.u, p.v, p.noise_re, p.noise_im, p.w)])
    a = ctx.chi2_image_multi(img, p.dxy, obs, [p.dRA], [p.dDec], [1.0], p.PA).item()
    b = ctx.chi2_image(img, p.dxy, obs, p.dRA, p.dDec, p.PA).item()
    assert a == b


def test_invalid_source_lists():
    ctx = Context(0)
    p = synth.small_image_problem(nxy=64, M=100, seed=1)
    d = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda")  # noqa: E731
    img, u, v = d(p.image), d(p.u), d(p.v)
    with pytest.raises(GalError):
        ctx.sample_image_multi(img, p.dxy, u, v, [], [], [])
    with pytest.raises(GalError):
        ctx.sample_image_multi(img, p.dxy, u, v, [0.0] * 17, [0.0] * 17, [1.0] * 17)
    with pytest.raises(GalError):
        ctx.sample_image_multi(img, p.dxy, u, v, [float("nan")], [0.0], [1.0])
