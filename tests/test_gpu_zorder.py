"""Observations registered in Z-order (gal_data_create_sorted_*): the same
chi-square as the input order up to the rounding of the summation order, the
same value on every registration, against the FP64 oracle at the tolerances
of the parity tests, and with the edge cases of plain registration."""
import ctypes as ct

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL_CHI2 = {torch.float64: 1e-12, torch.float32: 1e-6}
# the two orders add the same terms: only the summation order differs
TOL_ORDER = {torch.float64: 1e-12, torch.float32: 1e-6}
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
    return np.asarray(a, dtype=np.float32 if dt == torch.float32 else np.float64).astype(np.float64)


def synth():
    from paper_1709_06999_gb300 import synth as s
    return s


def _observation(q, model, dt):
    re, im = model.real + q.noise_re, model.imag + q.noise_im
    return [dev(a, dt) for a in (q.u, q.v, re, im, q.w)], re, im


@pytest.mark.parametrize("dt", DTYPES, ids=IDS)
def test_profile_window_through_l2(ctx, dt):
    """nxy 1024 with points to 0.45/dxy: the kept spectrum (929 x 465 nodes)
    is read through L2, the case the ordering is for."""
    s = synth()
    q = s.profile_problem(M=200_003)
    model = O.sample_profile(q.intensity, q.Rmin, q.dR, q.nxy, q.dxy, q.u, q.v, q.dRA, q.dDec,
                             q.PA, q.inc)
    arrs, re, im = _observation(q, model, dt)
    R = lambda a: rounded(a, dt)  # noqa: E731
    ref_vis = O.sample_profile(R(q.intensity), q.Rmin, q.dR, q.nxy, q.dxy, R(q.u), R(q.v),
                               q.dRA, q.dDec, q.PA, q.inc)
    ref = O.chi2(ref_vis, R(re), R(im), R(q.w))
    I_d = dev(q.intensity, dt)
    plain = ctx.register(*arrs)
    zo = ctx.register(*arrs, z_order=True)
    zo2 = ctx.register(*arrs, z_order=True)
    args = (q.Rmin, q.dR, q.nxy, q.dxy)
    geo = (q.inc, q.dRA, q.dDec, q.PA)
    a = ctx.chi2_profile(I_d, *args, plain, *geo).item()
    b = ctx.chi2_profile(I_d, *args, zo, *geo).item()
    c = ctx.chi2_profile(I_d, *args, zo2, *geo).item()
    assert abs(b - ref) <= TOL_CHI2[dt] * ref
    assert abs(b - a) <= TOL_ORDER[dt] * a
    assert b == c  # the order is the same on every registration
    # the copies are the library's own: the caller's arrays may change
    for t in arrs:
        t.fill_(0)
    assert ctx.chi2_profile(I_d, *args, zo, *geo).item() == b


@pytest.mark.parametrize("dt", DTYPES, ids=IDS)
def test_image_with_shared_window_and_batch(ctx, dt):
    from paper_1709_06999_gb300 import Request
    s = synth()
    p = s.small_image_problem(M=30_011)
    model = O.sample_image(p.image, p.dxy, p.u, p.v, p.dRA, p.dDec, p.PA)
    arrs, re, im = _observation(p, model, dt)
    R = lambda a: rounded(a, dt)  # noqa: E731
    ref = O.chi2(O.sample_image(R(p.image), p.dxy, R(p.u), R(p.v), p.dRA, p.dDec, p.PA),
                 R(re), R(im), R(p.w))
    img = dev(p.image, dt)
    zo = ctx.register(*arrs, z_order=True)
    b = ctx.chi2_image(img, p.dxy, zo, p.dRA, p.dDec, p.PA)
    assert abs(b.item() - ref) <= TOL_CHI2[dt] * ref
    reqs = [Request(zo, image=img, dxy=p.dxy, dRA=p.dRA, dDec=p.dDec, PA=p.PA + 0.1 * k)
            for k in range(5)]
    got = ctx.chi2_batch(reqs)
    single = torch.stack([ctx.chi2_image(img, p.dxy, zo, p.dRA, p.dDec, p.PA + 0.1 * k)
                          for k in range(5)])
    assert torch.equal(got, single)
    assert got[0] == b


@pytest.mark.parametrize("dt", DTYPES, ids=IDS)
def test_empty_and_non_finite(ctx, dt):
    s = synth()
    e = torch.empty(0, dtype=dt, device="cuda")
    zo = ctx.register(e, e, e, e, e, z_order=True)
    img = torch.zeros(64, 64, dtype=dt, device="cuda")
    assert ctx.chi2_image(img, 1e-7, zo, 0.0, 0.0, 0.0).item() == 0.0
    p = s.small_image_problem(M=1000)
    u = p.u.copy()
    u[17] = np.nan
    arrs = [dev(a, dt) for a in (u, p.v, p.noise_re, p.noise_im, p.w)]
    img = dev(p.image, dt)
    a = ctx.chi2_image(img, p.dxy, ctx.register(*arrs), p.dRA, p.dDec, p.PA).item()
    b = ctx.chi2_image(img, p.dxy, ctx.register(*arrs, z_order=True), p.dRA, p.dDec, p.PA).item()
    assert np.isnan(a) and np.isnan(b)


def test_invalid_arguments(ctx):
    from paper_1709_06999_gb300 import _native
    lib = _native.load()
    t = torch.zeros(16, dtype=torch.float32, device="cuda")
    h = ct.c_void_p()
    p = t.data_ptr()
    assert lib.gal_data_create_sorted_f32(ctx.handle, p, p, p, p, None, 16, None, ct.byref(h)) != 0
    assert lib.gal_data_create_sorted_f32(ctx.handle, p + 2, p, p, p, p, 16, None, ct.byref(h)) != 0
    assert lib.gal_data_create_sorted_f32(ctx.handle, p, p, p, p, p, -1, None, ct.byref(h)) != 0
    assert lib.gal_data_create_sorted_f32(None, p, p, p, p, p, 16, None, ct.byref(h)) != 0
    assert not h.value
    from paper_1709_06999_gb300.api import Observation
    with pytest.raises(ValueError):
        Observation(ctx, t, t, t, t, t, nu=t, z_order=True)
