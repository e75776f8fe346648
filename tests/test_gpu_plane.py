"""Primary beam and full-plane (complex-to-complex) spectrum against the oracle.

Both come in through the extended calls (gal_*_ex, options struct gal_opts):
the beam multiplies the model inside the row FFT, the full-plane path has its
own row kernel and an unfolded gather.  Tolerances as in test_gpu_parity.py
(normwise visibilities 1e-12 / 1e-5, relative chi-square 1e-12 / 1e-6); the
oracle is fed the same rounded inputs as the CUDA path.
"""
import ctypes as ct
import math

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL_VIS = {torch.float64: 1e-12, torch.float32: 1e-5}
TOL_CHI2 = {torch.float64: 1e-12, torch.float32: 1e-6}
DTYPES = [torch.float64, torch.float32]
IDS = ["f64", "f32"]


@pytest.fixture(scope="module")
def ctx():
    from paper_1709_06999_gb300 import Context
    c = Context(0)
    yield c
    c.check()
    c.close()


def synth():
    from paper_1709_06999_gb300 import synth as s
    return s


def dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def rounded(a, dt):
    return np.asarray(a, dtype=np.float32 if dt == torch.float32 else np.float64).astype(np.float64)


def as_complex(vis):
    v = vis.double().cpu().numpy()
    return v[:, 0] + 1j * v[:, 1]


def normwise(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def model_image(n, rng):
    s = synth()
    dxy = 0.02 * s.ARCSEC
    img = s.gaussian_image(n, dxy, 1.0, 0.1 * n * dxy, 0.06 * n * dxy, 0.4, 0.08 * n * dxy,
                           -0.05 * n * dxy)
    img += 0.01 * rng.standard_normal((n, n))
    img[rng.integers(0, n), rng.integers(0, n)] += 0.3
    return img, dxy


def min_size(dt):
    return 16 if dt == torch.float32 else 8


# ----------------------------------------------------------------------------
# full plane
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("dt", DTYPES, ids=IDS)
@pytest.mark.parametrize("n", [8, 16, 32, 64, 256, 1024])
def test_full_plane_sizes(ctx, dt, n):
    """Unpruned (points up to 1.3x the grid edge, clamped) at every transform
    structure, ragged M, both signs of u."""
    if n < min_size(dt):
        pytest.skip("below the full-plane size range of this precision")
    rng = np.random.default_rng(300 + n)
    img, dxy = model_image(n, rng)
    M = 2001 + 3 * n
    edge = (n / 2) / (n * dxy)
    u, v = synth().uv_loguniform(M, 0.01 * edge, 1.3 * edge, rng)
    u[:4] = [0.0, -0.0, -edge, edge]
    v[:4] = [0.0, 1.0 / (n * dxy), -edge, 0.5 * edge]
    kw = dict(dRA=0.2 * n * dxy / 64, dDec=-0.3 * n * dxy / 64, PA=0.9)
    ref = O.sample_image(rounded(img, dt), dxy, rounded(u, dt), rounded(v, dt), **kw,
                         full_plane=True)
    got = as_complex(ctx.sample_image(dev(img, dt), dxy, dev(u, dt), dev(v, dt), **kw,
                                      full_plane=True))
    assert normwise(got, ref) <= TOL_VIS[dt]


@pytest.mark.parametrize("dt", DTYPES, ids=IDS)
@pytest.mark.parametrize("PA", [0.0, math.pi / 2, 2.5])
def test_full_plane_pruned_chi2_and_vis(ctx, dt, PA):
    """A pruned window (ALMA-like coverage well inside the grid), chi2 and
    visibilities."""
    s = synth()
    p = s.small_image_problem(nxy=512, M=30011, seed=31)
    u, v = s.uv_loguniform(p.u.size, 1e4, 0.12 / p.dxy, np.random.default_rng(31))
    R = lambda a: rounded(a, dt)  # noqa: E731
    ref_vis = O.sample_image(R(p.image), p.dxy, R(u), R(v), p.dRA, p.dDec, PA, full_plane=True)
    re, im = ref_vis.real + p.noise_re, ref_vis.imag + p.noise_im
    ref = O.chi2(ref_vis, R(re), R(im), R(p.w))
    img, u_d, v_d = dev(p.image, dt), dev(u, dt), dev(v, dt)
    obs = ctx.register(u_d, v_d, dev(re, dt), dev(im, dt), dev(p.w, dt))
    chi2 = ctx.chi2_image(img, p.dxy, obs, p.dRA, p.dDec, PA, full_plane=True).item()
    assert abs(chi2 - ref) <= TOL_CHI2[dt] * ref
    got = as_complex(ctx.sample_image(img, p.dxy, u_d, v_d, p.dRA, p.dDec, PA, full_plane=True))
    assert normwise(got, ref_vis) <= TOL_VIS[dt]


@pytest.mark.parametrize("beam", [False, True], ids=["no_beam", "beam"])
def test_full_plane_unaligned_image(ctx, beam):
    """A float32 image 8- but not 16-byte aligned takes the full-plane row pass
    that loads pixels directly instead of staging rows with bulk copies."""
    s = synth()
    dt = torch.float32
    p = s.small_image_problem(nxy=256, M=15013, seed=39)
    kw = dict(pb_fwhm=0.5 * 256 * p.dxy) if beam else {}
    ref = O.sample_image(rounded(p.image, dt), p.dxy, rounded(p.u, dt), rounded(p.v, dt), p.dRA,
                         p.dDec, 0.8, full_plane=True, **kw)
    img = dev(p.image, dt)
    store = torch.empty(img.numel() + 2, dtype=dt, device="cuda")
    shifted = store[2:].view(img.shape)  # 8-byte offset from the 256-byte aligned allocation
    shifted.copy_(img)
    u_d, v_d = dev(p.u, dt), dev(p.v, dt)
    a = as_complex(ctx.sample_image(img, p.dxy, u_d, v_d, p.dRA, p.dDec, 0.8, full_plane=True, **kw))
    b = as_complex(ctx.sample_image(shifted, p.dxy, u_d, v_d, p.dRA, p.dDec, 0.8, full_plane=True,
                                    **kw))
    assert normwise(a, ref) <= TOL_VIS[dt]
    assert normwise(b, ref) <= TOL_VIS[dt]


@pytest.mark.parametrize("dt", DTYPES, ids=IDS)
def test_full_plane_agrees_with_half_plane(ctx, dt):
    """The paper's C2C versus R2C check, on the GPU: two independent spectrum
    paths give the same visibilities to rounding."""
    s = synth()
    p = s.small_image_problem(nxy=256, M=20011, seed=32)
    img, u_d, v_d = dev(p.image, dt), dev(p.u, dt), dev(p.v, dt)
    a = as_complex(ctx.sample_image(img, p.dxy, u_d, v_d, p.dRA, p.dDec, 1.2))
    b = as_complex(ctx.sample_image(img, p.dxy, u_d, v_d, p.dRA, p.dDec, 1.2, full_plane=True))
    assert normwise(b, a) <= 2 * TOL_VIS[dt]


@pytest.mark.parametrize("dt", DTYPES, ids=IDS)
def test_full_plane_profile(ctx, dt):
    """The sweep inside the full-plane row pass (inclined profile)."""
    s = synth()
    q = s.profile_problem(nxy=512, M=40011, nr=2048, seed=33)
    R = lambda a: rounded(a, dt)  # noqa: E731
    ref_vis = O.sample_profile(R(q.intensity), q.Rmin, q.dR, q.nxy, q.dxy, R(q.u), R(q.v),
                               q.dRA, q.dDec, q.PA, q.inc, full_plane=True)
    got = as_complex(ctx.sample_profile(dev(q.intensity, dt), q.Rmin, q.dR, q.nxy, q.dxy,
                                        dev(q.u, dt), dev(q.v, dt), q.inc, q.dRA, q.dDec, q.PA,
                                        full_plane=True))
    assert normwise(got, ref_vis) <= TOL_VIS[dt]


@pytest.mark.parametrize("dt", DTYPES, ids=IDS)
def test_full_plane_large_case(ctx, dt):
    """nxy = 4096, M = 5e6 (the benchmark workload) through the full plane:
    chi2 over all points, visibilities at every point."""
    s = synth()
    p = s.large_image_problem()
    R = lambda a: rounded(a, dt)  # noqa: E731
    Gf = O.full_spectrum(R(p.image))
    model = O.sample_full_spectrum(Gf, p.image.shape[0], p.dxy, R(p.u), R(p.v), p.dRA, p.dDec,
                                   p.PA)
    del Gf
    re, im = model.real + p.noise_re, model.imag + p.noise_im
    ref = O.chi2(model, R(re), R(im), R(p.w))
    img, u_d, v_d = dev(p.image, dt), dev(p.u, dt), dev(p.v, dt)
    obs = ctx.register(u_d, v_d, dev(re, dt), dev(im, dt), dev(p.w, dt))
    chi2 = ctx.chi2_image(img, p.dxy, obs, p.dRA, p.dDec, p.PA, full_plane=True).item()
    assert abs(chi2 - ref) <= TOL_CHI2[dt] * ref
    vis = as_complex(ctx.sample_image(img, p.dxy, u_d, v_d, p.dRA, p.dDec, p.PA,
                                      full_plane=True))
    assert normwise(vis, model) <= TOL_VIS[dt]


def test_full_plane_largest_size(ctx):
    """nxy = 8192 in float32 (the largest full-plane size), points over the
    whole grid: the window is the whole plane."""
    rng = np.random.default_rng(8193)
    s = synth()
    dt = torch.float32
    n, dxy = 8192, 0.001 * s.ARCSEC
    img = s.gaussian_image(n, dxy, 1.0, 0.3 * s.ARCSEC, 0.2 * s.ARCSEC, 1.0)
    img[4000, 5000] += 0.2
    u, v = s.uv_loguniform(20011, 1e4, 0.45 / dxy, rng)
    ref = O.sample_image(rounded(img, dt), dxy, rounded(u, dt), rounded(v, dt), 1e-7, 2e-7, 0.2,
                         full_plane=True)
    got = as_complex(ctx.sample_image(dev(img, dt), dxy, dev(u, dt), dev(v, dt), 1e-7, 2e-7, 0.2,
                                      full_plane=True))
    assert normwise(got, ref) <= TOL_VIS[dt]


# ----------------------------------------------------------------------------
# primary beam
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("dt", DTYPES, ids=IDS)
@pytest.mark.parametrize("n", [4, 8, 16, 32, 128, 512])
def test_beam_image_sizes(ctx, dt, n):
    """Every row-pass variant (the generic pass below the compile-time
    lengths, the staged one above) with a beam about as wide as the image."""
    rng = np.random.default_rng(400 + n)
    img, dxy = model_image(n, rng)
    M = 1501 + n
    edge = (n / 2) / (n * dxy)
    u, v = synth().uv_loguniform(M, 0.01 * edge, 0.9 * edge, rng)
    kw = dict(dRA=0.15 * n * dxy, dDec=-0.1 * n * dxy, PA=0.6)
    fwhm = 0.5 * n * dxy
    ref = O.sample_image(rounded(img, dt), dxy, rounded(u, dt), rounded(v, dt), **kw,
                         pb_fwhm=fwhm)
    got = as_complex(ctx.sample_image(dev(img, dt), dxy, dev(u, dt), dev(v, dt), **kw,
                                      pb_fwhm=fwhm))
    assert normwise(got, ref) <= TOL_VIS[dt]
    # the beam matters at this width
    plain = O.sample_image(rounded(img, dt), dxy, rounded(u, dt), rounded(v, dt), **kw)
    assert normwise(plain, ref) > 1e-2


@pytest.mark.parametrize("dt", DTYPES, ids=IDS)
def test_beam_image_chi2_and_unaligned(ctx, dt):
    """chi2 with a beam; an image that is not 16-byte aligned takes the
    row pass that loads pixels directly, with the same result."""
    s = synth()
    p = s.small_image_problem(nxy=256, M=20011, seed=34)
    fwhm = 0.6 * 256 * p.dxy
    R = lambda a: rounded(a, dt)  # noqa: E731
    ref_vis = O.sample_image(R(p.image), p.dxy, R(p.u), R(p.v), p.dRA, p.dDec, p.PA,
                             pb_fwhm=fwhm)
    re, im = ref_vis.real + p.noise_re, ref_vis.imag + p.noise_im
    ref = O.chi2(ref_vis, R(re), R(im), R(p.w))
    u_d, v_d = dev(p.u, dt), dev(p.v, dt)
    obs = ctx.register(u_d, v_d, dev(re, dt), dev(im, dt), dev(p.w, dt))
    img = dev(p.image, dt)
    chi2 = ctx.chi2_image(img, p.dxy, obs, p.dRA, p.dDec, p.PA, pb_fwhm=fwhm).item()
    assert abs(chi2 - ref) <= TOL_CHI2[dt] * ref
    store = torch.empty(img.numel() + 2, dtype=dt, device="cuda")
    shifted = store[2:].view(img.shape)  # 2 elements in: 8- (f32) or 16-byte (f64) offset
    shifted.copy_(img)
    a = ctx.sample_image(img, p.dxy, u_d, v_d, p.dRA, p.dDec, p.PA, pb_fwhm=fwhm)
    b = ctx.sample_image(shifted, p.dxy, u_d, v_d, p.dRA, p.dDec, p.PA, pb_fwhm=fwhm)
    assert normwise(as_complex(a), ref_vis) <= TOL_VIS[dt]
    assert normwise(as_complex(b), ref_vis) <= TOL_VIS[dt]


@pytest.mark.parametrize("dt", DTYPES, ids=IDS)
def test_beam_profile_case(ctx, dt):
    """The inclined profile case (nxy = 1024, M = 1e6) through a beam that is
    evaluated on the sky, not on the deprojected disc."""
    s = synth()
    q = s.profile_problem()
    fwhm = 1.5 * s.ARCSEC
    R = lambda a: rounded(a, dt)  # noqa: E731
    ref_vis = O.sample_profile(R(q.intensity), q.Rmin, q.dR, q.nxy, q.dxy, R(q.u), R(q.v),
                               q.dRA, q.dDec, q.PA, q.inc, pb_fwhm=fwhm)
    re, im = ref_vis.real + q.noise_re, ref_vis.imag + q.noise_im
    ref = O.chi2(ref_vis, R(re), R(im), R(q.w))
    I_d, u_d, v_d = dev(q.intensity, dt), dev(q.u, dt), dev(q.v, dt)
    obs = ctx.register(u_d, v_d, dev(re, dt), dev(im, dt), dev(q.w, dt))
    chi2 = ctx.chi2_profile(I_d, q.Rmin, q.dR, q.nxy, q.dxy, obs, q.inc, q.dRA, q.dDec, q.PA,
                            pb_fwhm=fwhm).item()
    assert abs(chi2 - ref) <= TOL_CHI2[dt] * ref
    got = as_complex(ctx.sample_profile(I_d, q.Rmin, q.dR, q.nxy, q.dxy, u_d, v_d, q.inc, q.dRA,
                                        q.dDec, q.PA, pb_fwhm=fwhm))
    assert normwise(got, ref_vis) <= TOL_VIS[dt]


@pytest.mark.parametrize("dt", DTYPES, ids=IDS)
def test_beam_with_full_plane(ctx, dt):
    s = synth()
    p = s.small_image_problem(nxy=512, M=25013, seed=35)
    fwhm = 0.4 * 512 * p.dxy
    R = lambda a: rounded(a, dt)  # noqa: E731
    kw = dict(dRA=3e-7, dDec=-2e-7, PA=2.1)
    ref_vis = O.sample_image(R(p.image), p.dxy, R(p.u), R(p.v), **kw, pb_fwhm=fwhm,
                             full_plane=True)
    re, im = ref_vis.real + p.noise_re, ref_vis.imag + p.noise_im
    ref = O.chi2(ref_vis, R(re), R(im), R(p.w))
    img, u_d, v_d = dev(p.image, dt), dev(p.u, dt), dev(p.v, dt)
    obs = ctx.register(u_d, v_d, dev(re, dt), dev(im, dt), dev(p.w, dt))
    chi2 = ctx.chi2_image(img, p.dxy, obs, **kw, pb_fwhm=fwhm, full_plane=True).item()
    assert abs(chi2 - ref) <= TOL_CHI2[dt] * ref
    got = as_complex(ctx.sample_image(img, p.dxy, u_d, v_d, **kw, pb_fwhm=fwhm, full_plane=True))
    assert normwise(got, ref_vis) <= TOL_VIS[dt]


@pytest.mark.parametrize("dt", DTYPES, ids=IDS)
def test_wide_beam_is_no_beam_bitwise(ctx, dt):
    """A beam far wider than the image rounds to exactly 1 at every pixel, so
    the result is bitwise the plain call's (same kernels, factors of 1)."""
    s = synth()
    p = s.small_image_problem(nxy=256, M=10007, seed=36)
    img, u_d, v_d = dev(p.image, dt), dev(p.u, dt), dev(p.v, dt)
    a = ctx.sample_image(img, p.dxy, u_d, v_d, p.dRA, p.dDec, p.PA)
    b = ctx.sample_image(img, p.dxy, u_d, v_d, p.dRA, p.dDec, p.PA, pb_fwhm=1e6)
    assert torch.equal(a, b)


# ----------------------------------------------------------------------------
# the options struct itself
# ----------------------------------------------------------------------------
def test_null_options_equal_plain_call(ctx):
    s = synth()
    p = s.small_image_problem(nxy=128, M=5003, seed=37)
    dt = torch.float32
    img, u_d, v_d = dev(p.image, dt), dev(p.u, dt), dev(p.v, dt)
    a = ctx.sample_image(img, p.dxy, u_d, v_d, p.dRA, p.dDec, p.PA)
    b = torch.empty_like(a)
    st = ctx._stream()
    rc = ctx.lib.gal_sample_image_ex_f32(ctx.handle, img.data_ptr(), 128, p.dxy, p.dRA, p.dDec,
                                         p.PA, None, u_d.numel(), u_d.data_ptr(), v_d.data_ptr(),
                                         b.data_ptr(), st)
    assert rc == 0
    assert torch.equal(a, b)


def test_invalid_options_launch_nothing(ctx):
    from paper_1709_06999_gb300 import GalError
    from paper_1709_06999_gb300._native import GalOpts
    s = synth()
    p = s.small_image_problem(nxy=64, M=1001, seed=38)
    u32, v32 = dev(p.u, torch.float32), dev(p.v, torch.float32)
    img32 = dev(p.image, torch.float32)
    n0 = ctx.launch_count()
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(GalError):
            ctx.sample_image(img32, p.dxy, u32, v32, pb_fwhm=bad)
    small = dev(p.image[28:36, 28:36], torch.float32)  # nxy = 8: below the f32 full-plane range
    with pytest.raises(GalError):
        ctx.sample_image(small, p.dxy, u32, v32, full_plane=True)
    out = torch.empty((u32.numel(), 2), dtype=torch.float32, device="cuda")
    opts = GalOpts(0.0, 2)
    rc = ctx.lib.gal_sample_image_ex_f32(ctx.handle, img32.data_ptr(), 64, p.dxy, 0.0, 0.0, 0.0,
                                         ct.byref(opts), u32.numel(), u32.data_ptr(),
                                         v32.data_ptr(), out.data_ptr(), ctx._stream())
    assert rc == -1
    big = torch.zeros((8192, 8192), dtype=torch.float64, device="cuda")
    u64, v64 = dev(p.u, torch.float64), dev(p.v, torch.float64)
    with pytest.raises(GalError):  # float64 full plane stops at 4096
        ctx.sample_image(big, p.dxy, u64, v64, full_plane=True)
    assert ctx.launch_count() == n0
