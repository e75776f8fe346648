"""CUDA path against the FP64 oracle, element by element, through the C ABI.

Tolerances (normwise for visibilities: max_k |dV_k| / max_k |V_k|; relative
for chi-square):
    float64 path: visibilities 1e-12, chi2 1e-12
    float32 path: visibilities 1e-5,  chi2 1e-6
For the float32 path the oracle is fed the very same float32-rounded inputs,
promoted to float64, so the error measured is the path's own arithmetic.
"""
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


def dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def rounded(a, dt):
    """The values the CUDA path sees, as float64 for the oracle."""
    return np.asarray(a, dtype=np.float32 if dt == torch.float32 else np.float64).astype(np.float64)


def as_complex(vis):
    v = vis.double().cpu().numpy()
    return v[:, 0] + 1j * v[:, 1]


def normwise(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def synth():
    from paper_1709_06999_gb300 import synth as s
    return s


def random_image(n, rng):
    s = synth()
    dxy = 0.02 * s.ARCSEC
    img = s.gaussian_image(n, dxy, 1.0, 0.12 * n / 64 * dxy * 20, 0.07 * n / 64 * dxy * 20, 0.4,
                           0.1 * n * dxy, -0.05 * n * dxy)
    img += 0.01 * rng.standard_normal((n, n))
    img[rng.integers(0, n), rng.integers(0, n)] += 0.3
    return img, dxy


# ----------------------------------------------------------------------------
# small sizes: every FFT stage structure, ragged M, off-grid points
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("dt", DTYPES, ids=IDS)
@pytest.mark.parametrize("n", [4, 8, 16, 32, 64, 128, 256, 512])
def test_sample_image_sizes(ctx, dt, n):
    rng = np.random.default_rng(100 + n)
    img, dxy = random_image(n, rng)
    M = 1001 + n
    edge = (n / 2) / (n * dxy)        # |u| of the last grid column
    u, v = synth().uv_loguniform(M, 0.01 * edge, 1.3 * edge, rng)   # some beyond the grid
    u[:3] = [0.0, -0.0, edge]
    v[:3] = [0.0, 1.0 / (n * dxy), -edge]
    kw = dict(dRA=0.3 * n * dxy / 64, dDec=-0.2 * n * dxy / 64, PA=0.7)
    ref = O.sample_image(rounded(img, dt), dxy, rounded(u, dt), rounded(v, dt), **kw)
    got = as_complex(ctx.sample_image(dev(img, dt), dxy, dev(u, dt), dev(v, dt), **kw))
    assert normwise(got, ref) <= TOL_VIS[dt]


@pytest.mark.parametrize("dt", DTYPES, ids=IDS)
@pytest.mark.parametrize("PA", [0.0, math.pi / 2, 2.5, -1.0])
def test_sample_image_position_angles(ctx, dt, PA):
    s = synth()
    p = s.small_image_problem(nxy=128, M=4003, seed=7)
    ref = O.sample_image(rounded(p.image, dt), p.dxy, rounded(p.u, dt), rounded(p.v, dt),
                         p.dRA, p.dDec, PA)
    got = as_complex(ctx.sample_image(dev(p.image, dt), p.dxy, dev(p.u, dt), dev(p.v, dt),
                                      p.dRA, p.dDec, PA))
    assert normwise(got, ref) <= TOL_VIS[dt]


# ----------------------------------------------------------------------------
# the small image case (nxy=256, M=1e4) and the profile case (nxy=1024, M=1e6)
# ----------------------------------------------------------------------------
def observed(model, p, dt):
    re = model.real + p.noise_re
    im = model.imag + p.noise_im
    return re, im


@pytest.mark.parametrize("dt", DTYPES, ids=IDS)
def test_small_image_case(ctx, dt):
    s = synth()
    p = s.small_image_problem()
    model = O.sample_image(p.image, p.dxy, p.u, p.v, p.dRA, p.dDec, p.PA)
    re, im = observed(model, p, dt)
    img_d, u_d, v_d = dev(p.image, dt), dev(p.u, dt), dev(p.v, dt)
    obs = ctx.register(u_d, v_d, dev(re, dt), dev(im, dt), dev(p.w, dt))
    chi2 = ctx.chi2_image(img_d, p.dxy, obs, p.dRA, p.dDec, p.PA).item()
    R = lambda a: rounded(a, dt)  # noqa: E731
    ref_vis = O.sample_image(R(p.image), p.dxy, R(p.u), R(p.v), p.dRA, p.dDec, p.PA)
    ref = O.chi2(ref_vis, R(re), R(im), R(p.w))
    assert abs(chi2 - ref) <= TOL_CHI2[dt] * ref
    got = as_complex(ctx.sample_image(img_d, p.dxy, u_d, v_d, p.dRA, p.dDec, p.PA))
    assert normwise(got, ref_vis) <= TOL_VIS[dt]


@pytest.mark.parametrize("dt", DTYPES, ids=IDS)
def test_profile_case(ctx, dt):
    s = synth()
    q = s.profile_problem()
    model = O.sample_profile(q.intensity, q.Rmin, q.dR, q.nxy, q.dxy, q.u, q.v, q.dRA, q.dDec,
                             q.PA, q.inc)
    re, im = observed(model, q, dt)
    R = lambda a: rounded(a, dt)  # noqa: E731
    ref_vis = O.sample_profile(R(q.intensity), q.Rmin, q.dR, q.nxy, q.dxy, R(q.u), R(q.v),
                               q.dRA, q.dDec, q.PA, q.inc)
    ref = O.chi2(ref_vis, R(re), R(im), R(q.w))
    I_d, u_d, v_d = dev(q.intensity, dt), dev(q.u, dt), dev(q.v, dt)
    obs = ctx.register(u_d, v_d, dev(re, dt), dev(im, dt), dev(q.w, dt))
    chi2 = ctx.chi2_profile(I_d, q.Rmin, q.dR, q.nxy, q.dxy, obs, q.inc, q.dRA, q.dDec,
                            q.PA).item()
    assert abs(chi2 - ref) <= TOL_CHI2[dt] * ref
    got = as_complex(ctx.sample_profile(I_d, q.Rmin, q.dR, q.nxy, q.dxy, u_d, v_d, q.inc, q.dRA,
                                        q.dDec, q.PA))
    assert normwise(got, ref_vis) <= TOL_VIS[dt]


@pytest.mark.parametrize("dt", DTYPES, ids=IDS)
@pytest.mark.parametrize("inc_deg", [0.0, 45.0, 80.0])
def test_sweep(ctx, dt, inc_deg):
    s = synth()
    q = s.profile_problem(nxy=256, M=1, nr=3000, dxy=0.02 * s.ARCSEC)
    inc = inc_deg * s.DEG
    got = ctx.sweep(dev(q.intensity, dt), q.Rmin, q.dR, q.nxy, q.dxy, inc).double().cpu().numpy()
    ref = O.sweep(rounded(q.intensity, dt), q.Rmin, q.dR, q.nxy, q.dxy, inc)
    tol = 1e-12 if dt == torch.float64 else 2e-6
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))


@pytest.mark.parametrize("dt", DTYPES, ids=IDS)
def test_profile_equals_image_of_sweep(ctx, dt):
    """sample_profile (sweep fused into the FFT) equals sample_image of the swept
    image bit for bit: the same pixel values enter the same FFT (Sect. 5 reports
    the two functions agree to machine precision)."""
    s = synth()
    q = s.profile_problem(nxy=512, M=5003, nr=2048, dxy=0.01 * s.ARCSEC)
    I_d, u_d, v_d = dev(q.intensity, dt), dev(q.u, dt), dev(q.v, dt)
    img = ctx.sweep(I_d, q.Rmin, q.dR, q.nxy, q.dxy, q.inc)
    a = ctx.sample_profile(I_d, q.Rmin, q.dR, q.nxy, q.dxy, u_d, v_d, q.inc, q.dRA, q.dDec, 0.3)
    b = ctx.sample_image(img, q.dxy, u_d, v_d, q.dRA, q.dDec, 0.3)
    assert torch.equal(a, b)


# ----------------------------------------------------------------------------
# invariants on the GPU
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("dt", DTYPES, ids=IDS)
def test_hermitian_bitwise(ctx, dt):
    s = synth()
    p = s.small_image_problem(nxy=256, M=2000, seed=3)
    img = dev(p.image, dt)
    u, v = dev(p.u, dt), dev(p.v, dt)
    a = ctx.sample_image(img, p.dxy, u, v, p.dRA, p.dDec, 1.2)
    b = ctx.sample_image(img, p.dxy, -u, -v, p.dRA, p.dDec, 1.2)
    assert torch.equal(a[:, 0], b[:, 0]) and torch.equal(a[:, 1], -b[:, 1])


@pytest.mark.parametrize("dt", DTYPES, ids=IDS)
def test_chi2_repeatable_and_zero_at_model(ctx, dt):
    s = synth()
    p = s.small_image_problem(nxy=256, M=30011, seed=4)
    img = dev(p.image, dt)
    u, v = dev(p.u, dt), dev(p.v, dt)
    vis = ctx.sample_image(img, p.dxy, u, v, p.dRA, p.dDec, p.PA)
    obs = ctx.register(u, v, vis[:, 0].contiguous(), vis[:, 1].contiguous(), dev(p.w, dt))
    c1 = ctx.chi2_image(img, p.dxy, obs, p.dRA, p.dDec, p.PA).item()
    c2 = ctx.chi2_image(img, p.dxy, obs, p.dRA, p.dDec, p.PA).item()
    assert c1 == 0.0 and c2 == 0.0
    obs2 = ctx.register(u, v, (vis[:, 0] + 1).contiguous(), vis[:, 1].contiguous(), dev(p.w, dt))
    r = [ctx.chi2_image(img, p.dxy, obs2, p.dRA, p.dDec, p.PA).item() for _ in range(3)]
    assert r[0] == r[1] == r[2]
    assert abs(r[0] - rounded(p.w, dt).sum()) <= 1e-6 * r[0]


@pytest.mark.parametrize("dt", DTYPES, ids=IDS)
def test_pruning_is_exact(ctx, dt):
    """Adding one far uv point widens the kept part of the spectrum (here to the
    whole half plane).  Pruning drops no term, so the other points'
    visibilities agree to rounding (the pruned transform evaluates its kept
    outputs with a different summation order, so not bit for bit)."""
    s = synth()
    p = s.small_image_problem(nxy=512, M=3000, seed=9)
    p.u *= 0.1
    p.v *= 0.1
    img = dev(p.image, dt)
    a = ctx.sample_image(img, p.dxy, dev(p.u, dt), dev(p.v, dt), p.dRA, p.dDec, 0.4)
    far = 0.49 / p.dxy
    b = ctx.sample_image(img, p.dxy, dev(np.append(p.u, far), dt), dev(np.append(p.v, -far), dt),
                         p.dRA, p.dDec, 0.4)
    tol = 1e-14 if dt == torch.float64 else 1e-6
    assert normwise(as_complex(a), as_complex(b[:-1])) <= tol


def test_image_alignment_paths_agree(ctx):
    """A 16-byte aligned float32 image takes the TMA-staged row pass, one that
    is only 8-byte aligned the register-load row pass; both match the oracle.
    (float64 images are always 16-byte aligned.)"""
    dt = torch.float32
    s = synth()
    p = s.small_image_problem(nxy=1024, M=7001, seed=12)
    flat = torch.zeros(1024 * 1024 + 2, dtype=dt, device="cuda")
    shifted = flat[2:].view(1024, 1024)
    shifted.copy_(dev(p.image, dt))
    u, v = dev(p.u, dt), dev(p.v, dt)
    ref = O.sample_image(rounded(p.image, dt), p.dxy, rounded(p.u, dt), rounded(p.v, dt),
                         p.dRA, p.dDec, 0.5)
    a = as_complex(ctx.sample_image(dev(p.image, dt), p.dxy, u, v, p.dRA, p.dDec, 0.5))
    b = as_complex(ctx.sample_image(shifted, p.dxy, u, v, p.dRA, p.dDec, 0.5))
    assert normwise(a, ref) <= TOL_VIS[dt]
    assert normwise(b, ref) <= TOL_VIS[dt]


# ----------------------------------------------------------------------------
# edge cases
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("dt", DTYPES, ids=IDS)
def test_host_async_pipeline_equals_host_calls(ctx, dt):
    """Pipelined host-buffer calls (copy of call k+1 overlapping the compute of
    call k, two staging buffers in turn) give bitwise the synchronous
    host-buffer results, for three host images used in rotation."""
    s = synth()
    p = s.small_image_problem(nxy=512, M=20011, seed=41)
    obs = ctx.register(dev(p.u, dt), dev(p.v, dt), dev(p.noise_re, dt), dev(p.noise_im, dt),
                       dev(p.w, dt))
    imgs = [torch.as_tensor(p.image * (1.0 + 0.1 * k), dtype=dt).pin_memory() for k in range(3)]
    n = 11
    want = [ctx.chi2_image_host(imgs[k % 3], p.dxy, obs, p.dRA, p.dDec, 0.2 * k) for k in range(n)]
    out = torch.full((n,), float("nan"), dtype=torch.float64).pin_memory()
    for k in range(n):
        ctx.chi2_image_host_async(imgs[k % 3], p.dxy, obs, out, k, p.dRA, p.dDec, 0.2 * k)
    torch.cuda.current_stream().synchronize()
    assert out.tolist() == want
    # a larger image regrows the staging buffers after their last use
    big = torch.as_tensor(np.pad(p.image, 256), dtype=dt).pin_memory()
    ref = ctx.chi2_image_host(big, p.dxy, obs, p.dRA, p.dDec, 0.3)
    ctx.chi2_image_host_async(big, p.dxy, obs, out, 0, p.dRA, p.dDec, 0.3)
    ctx.chi2_image_host_async(imgs[0], p.dxy, obs, out, 1, p.dRA, p.dDec, 0.0)
    torch.cuda.current_stream().synchronize()
    assert out[0].item() == ref and out[1].item() == want[0]


@pytest.mark.parametrize("dt", DTYPES, ids=IDS)
def test_empty_observation(ctx, dt):
    e = torch.empty(0, dtype=dt, device="cuda")
    obs = ctx.register(e, e, e, e, e)
    img = torch.rand(64, 64, dtype=dt, device="cuda")
    out = torch.full((), 7.0, dtype=torch.float64, device="cuda")
    assert ctx.chi2_image(img, 1e-7, obs, out=out).item() == 0.0
    assert ctx.sample_image(img, 1e-7, e, e).shape == (0, 2)


@pytest.mark.parametrize("dt", DTYPES, ids=IDS)
def test_nan_propagates(ctx, dt):
    img = torch.rand(32, 32, dtype=dt, device="cuda")
    u = torch.tensor([1e5, float("nan"), 2e5, 3e5], dtype=dt, device="cuda")
    v = torch.tensor([0.0, 1e5, float("nan"), 1e4], dtype=dt, device="cuda")
    vis = ctx.sample_image(img, 1e-7, u, v).cpu()
    assert torch.isnan(vis[1]).all() and torch.isnan(vis[2]).all()
    assert torch.isfinite(vis[0]).all() and torch.isfinite(vis[3]).all()


def test_invalid_arguments(ctx):
    from paper_1709_06999_gb300 import GalError
    img = torch.rand(48, 48, device="cuda")
    u = torch.zeros(4, device="cuda")
    with pytest.raises(GalError):
        ctx.sample_image(img, 1e-7, u, u)                       # not a power of two
    with pytest.raises(GalError):
        ctx.sample_image(torch.rand(64, 64, device="cuda"), 0.0, u, u)    # dxy <= 0
    I = torch.rand(16, device="cuda")
    with pytest.raises(GalError):
        ctx.sweep(I, 0.0, 1e-8, 64, 1e-7, inc=math.pi / 2)      # |inc| >= pi/2
    with pytest.raises(GalError):
        ctx.sweep(I[:1], 0.0, 1e-8, 64, 1e-7)                   # nr < 2
    with pytest.raises(GalError):
        ctx.sweep(I, 0.0, -1e-8, 64, 1e-7)                      # dR <= 0
    obs64 = ctx.register(*(torch.zeros(4, dtype=torch.float64, device="cuda") for _ in range(5)))
    with pytest.raises(GalError):
        ctx.chi2_image(torch.rand(64, 64, device="cuda"), 1e-7, obs64)   # precision mismatch
    with pytest.raises(GalError):
        ctx.sample_image(torch.empty(16384, 16384, device="cuda"), 1e-7, u, u)  # nxy > 8192


def test_workspace_regrowth_and_counters(ctx):
    s = synth()
    before = ctx.launch_count()
    for n in (64, 1024, 64, 256):
        p = s.small_image_problem(nxy=n, M=999, seed=n)
        ref = O.sample_image(p.image, p.dxy, p.u, p.v, p.dRA, p.dDec, p.PA)
        got = as_complex(ctx.sample_image(dev(p.image, torch.float64), p.dxy,
                                          dev(p.u, torch.float64), dev(p.v, torch.float64),
                                          p.dRA, p.dDec, p.PA))
        assert normwise(got, ref) <= 1e-12
    assert ctx.launch_count() - before >= 4 * 4
    ctx.set_stage_timing(True)
    p = s.small_image_problem(nxy=256, M=5000, seed=1)
    obs = ctx.register(*(dev(a, torch.float32) for a in (p.u, p.v, p.noise_re, p.noise_im, p.w)))
    for _ in range(3):
        ctx.chi2_image(dev(p.image, torch.float32), p.dxy, obs)
    times = ctx.stage_times()
    ctx.set_stage_timing(False)
    assert [n for _, n in times] == [1, 3, 3, 3]
    assert all(ms > 0 for ms, n in times if n)


def test_hbm_budget():
    """A context's workspace limit: growth past it is GAL_E_NOMEM with the
    workspace unchanged and nothing evaluated; calls within it still run."""
    from paper_1709_06999_gb300 import Context, GalError
    s = synth()
    c = Context(0)
    p = s.small_image_problem(nxy=64, M=2001, seed=3)
    obs = c.register(*(dev(a, torch.float32) for a in (p.u, p.v, p.noise_re, p.noise_im, p.w)))
    small = dev(p.image, torch.float32)
    a = c.chi2_image(small, p.dxy, obs).item()
    held = c.workspace_bytes()
    c.set_hbm_budget(held)
    assert c.chi2_image(small, p.dxy, obs).item() == a  # no growth needed
    big = torch.zeros(1024, 1024, dtype=torch.float32, device="cuda")
    out = torch.full((), -1.0, dtype=torch.float64, device="cuda")
    u, v = dev(p.u, torch.float32), dev(p.v, torch.float32)
    vis = torch.full((u.numel(), 2), -1.0, dtype=torch.float32, device="cuda")
    launches = c.launch_count()
    with pytest.raises(GalError, match="status -2"):
        c.chi2_image(big, p.dxy, obs, out=out)
    with pytest.raises(GalError, match="status -2"):
        c.chi2_image(big, p.dxy, obs, out=out, pb_fwhm=1e-4)
    with pytest.raises(GalError, match="status -2"):
        c.sample_image(big, p.dxy, u, v, out=vis)
    assert c.launch_count() == launches  # nothing was enqueued
    assert out.item() == -1.0 and bool((vis == -1.0).all()) and c.workspace_bytes() == held
    c.set_hbm_budget(0)
    c.chi2_image(big, p.dxy, obs, out=out)
    assert out.item() != -1.0 and c.workspace_bytes() > held
    c.close()


# ----------------------------------------------------------------------------
# full size, in the benchmark's launch configuration (registered observation,
# chi2_image; float32 is the bench line, float64 its plain FP64 comparison):
# chi2 over all 5e6 points and visibilities at sampled and all points, against
# the oracle
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("dt", DTYPES, ids=IDS)
def test_large_image_case(ctx, dt):
    s = synth()
    p = s.large_image_problem()
    R = lambda a: rounded(a, dt)  # noqa: E731
    G = O.half_spectrum(R(p.image))
    model = O.sample_spectrum(G, p.image.shape[0], p.dxy, R(p.u), R(p.v), p.dRA, p.dDec, p.PA)
    re, im = model.real + p.noise_re, model.imag + p.noise_im
    ref = O.chi2(model, R(re), R(im), R(p.w))
    img = dev(p.image, dt)
    u_d, v_d = dev(p.u, dt), dev(p.v, dt)
    obs = ctx.register(u_d, v_d, dev(re, dt), dev(im, dt), dev(p.w, dt))
    chi2 = ctx.chi2_image(img, p.dxy, obs, p.dRA, p.dDec, p.PA).item()
    assert abs(chi2 - ref) <= TOL_CHI2[dt] * ref
    vis = as_complex(ctx.sample_image(img, p.dxy, u_d, v_d, p.dRA, p.dDec, p.PA))
    idx = np.random.default_rng(0).choice(p.u.size, 20000, replace=False)
    assert normwise(vis[idx], model[idx]) <= TOL_VIS[dt]
    assert normwise(vis, model) <= TOL_VIS[dt]


@pytest.mark.parametrize("dt", DTYPES, ids=IDS)
def test_largest_image_size(ctx, dt):
    """nxy = 8192, the largest supported size, with points over the whole grid."""
    rng = np.random.default_rng(8192)
    s = synth()
    n, dxy = 8192, 0.001 * s.ARCSEC
    img = s.gaussian_image(n, dxy, 1.0, 0.3 * s.ARCSEC, 0.2 * s.ARCSEC, 1.0)
    img[4000, 5000] += 0.2
    u, v = s.uv_loguniform(20011, 1e4, 0.45 / dxy, rng)
    ref = O.sample_image(rounded(img, dt), dxy, rounded(u, dt), rounded(v, dt), 1e-7, 2e-7, 0.2)
    got = as_complex(ctx.sample_image(dev(img, dt), dxy, dev(u, dt), dev(v, dt), 1e-7, 2e-7, 0.2))
    assert normwise(got, ref) <= TOL_VIS[dt]
