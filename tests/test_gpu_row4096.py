"""The float row pass of 4096-pixel images against the FP64 oracle, on every
branch it takes (GPU).

Rows of that length run one kernel whose pruned last stage is evaluated in
registers and warp shuffles when the kept window has at most 64 columns, and
by the generic Stockham last stage otherwise (wider pruned windows, or the
whole half spectrum).  The width follows from the uv extent: Kc = floor(e) + 4
columns for a largest grid offset of e = max|uv| nxy dxy cells (Sect. 3.3 and
App. D: the bilinear stencil plus a margin), so extents of 60.5 and 61.5
cells sit on the two sides of the boundary.  Each case checks the sampled
visibilities (Sect. 3.2) and chi-square (Sect. 3.1) against the oracle within
the float32 gates, and a batch of the same request against the single call
bit for bit (both run the same kernel).
"""
import math

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N = 4096
TOL_VIS = 1e-5
TOL_CHI2 = 1e-6
# (largest grid offset in cells, expected kept columns)
CASES = [(60.5, 64), (61.5, 65), (200.5, 204), (900.5, 904), (2047.0, 2049)]


def r32(a):
    return np.asarray(a, np.float32).astype(np.float64)


@pytest.fixture(scope="module")
def image():
    from paper_1709_06999_gb300 import synth
    dxy = 0.002 * synth.ARCSEC
    img = synth.large_image(N, dxy, np.random.default_rng(7))
    return img.astype(np.float32).astype(np.float64), dxy


def points(e, dxy, M, seed):
    """M points with radius uniform below e cells (one exactly at e)."""
    rng = np.random.default_rng(seed)
    rmax = e / (N * dxy)
    r = rmax * np.sqrt(rng.uniform(0.0, 1.0, M))
    th = rng.uniform(0.0, 2.0 * math.pi, M)
    r[0], th[0] = rmax * (1.0 - 1e-7), 0.3
    u, v = r * np.cos(th), r * np.sin(th)
    w = rng.uniform(0.5, 2.0, M)
    return u, v, w, rng


@pytest.mark.parametrize("e,kc", CASES, ids=[f"Kc{kc}" for _, kc in CASES])
def test_row_pass_4096_branches(image, e, kc):
    from paper_1709_06999_gb300 import Context, Request
    img, dxy = image
    u, v, w, rng = points(e, dxy, 20011, seed=int(e))
    S = N * dxy
    ext = math.sqrt(float(np.max(r32(u) ** 2 + r32(v) ** 2))) * S
    assert math.floor(ext) + 4 == kc or (kc == N // 2 + 1 and ext >= N // 2 - 4)
    dRA, dDec, PA = 0.031 * math.pi / 648000, -0.017 * math.pi / 648000, 0.7
    ref = O.sample_image(img, dxy, r32(u), r32(v), dRA, dDec, PA)
    re = (ref.real + rng.normal(0.0, 1.0, ref.shape) / np.sqrt(w)).astype(np.float32)
    im = (ref.imag + rng.normal(0.0, 1.0, ref.shape) / np.sqrt(w)).astype(np.float32)
    chi2_ref = O.chi2(ref, r32(re), r32(im), r32(w))
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")  # noqa: E731
    ctx = Context(0)
    gi, gu, gv = dev(img), dev(u), dev(v)
    vis = ctx.sample_image(gi, dxy, gu, gv, dRA, dDec, PA).double().cpu().numpy()
    V = vis[:, 0] + 1j * vis[:, 1]
    err = np.max(np.abs(V - ref)) / np.max(np.abs(ref))
    assert err <= TOL_VIS, err
    obs = ctx.register(gu, gv, dev(re), dev(im), dev(w))
    single = ctx.chi2_image(gi, dxy, obs, dRA, dDec, PA).item()
    assert abs(single - chi2_ref) <= TOL_CHI2 * chi2_ref, (single, chi2_ref)
    batch = ctx.chi2_batch([Request(obs, image=gi, dxy=dxy, dRA=dRA, dDec=dDec, PA=PA)] * 2)
    assert batch.cpu().numpy().tolist() == [single] * 2
    ctx.check()
    obs.close()
    ctx.close()


@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_small_batches_of_the_large_case_equal_single_calls(n):
    """A batch runs each request's gather as virtual blocks, up to four per
    launched block but never more than the launch has requests; whatever the
    count, every request's chi-square is its single call's, bit for bit."""
    from paper_1709_06999_gb300 import Context, Request, synth
    p = synth.large_image_problem(M=2_000_003, seed=9)  # 3 whole rounds, a remainder, a tail
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")  # noqa: E731
    ctx = Context(0)
    obs = ctx.register(dev(p.u), dev(p.v), dev(p.noise_re), dev(p.noise_im), dev(p.w))
    img = dev(p.image)
    rng = np.random.default_rng(n)
    reqs = []
    for k in range(n):
        a, b = rng.uniform(-0.1, 0.1, 2) * math.pi / 648000
        reqs.append(Request(obs, image=img * float(1.0 + 0.01 * k), dxy=p.dxy, dRA=float(a),
                            dDec=float(b), PA=float(rng.uniform(0.0, math.pi))))
    got = ctx.chi2_batch(reqs).cpu().numpy().tolist()
    want = [ctx.chi2_image(r.image, r.dxy, obs, r.dRA, r.dDec, r.PA).item() for r in reqs]
    assert got == want
    ctx.check()
    obs.close()
    ctx.close()


@pytest.mark.parametrize("e,kc", [(60.5, 64), (200.5, 204)], ids=["Kc64", "Kc204"])
def test_row_pass_4096_with_primary_beam(image, e, kc):
    """The same row pass with the primary beam applied as pixels enter
    registers (Sect. 2.1: the model times the antenna pattern, here a Gaussian
    of FWHM about a third of the field), against the oracle; a batch of the
    same request is bitwise its single call."""
    from paper_1709_06999_gb300 import Context, Request
    img, dxy = image
    u, v, w, rng = points(e, dxy, 20011, seed=int(e) + 1)
    fwhm = 0.35 * N * dxy
    dRA, dDec, PA = 0.05 * math.pi / 648000, 0.02 * math.pi / 648000, 1.1
    ref = O.sample_image(img, dxy, r32(u), r32(v), dRA, dDec, PA, pb_fwhm=fwhm)
    plain = O.sample_image(img, dxy, r32(u), r32(v), dRA, dDec, PA)
    assert np.max(np.abs(plain - ref)) > 1e-3 * np.max(np.abs(ref))   # the beam matters
    re = (ref.real + rng.normal(0.0, 1.0, ref.shape) / np.sqrt(w)).astype(np.float32)
    im = (ref.imag + rng.normal(0.0, 1.0, ref.shape) / np.sqrt(w)).astype(np.float32)
    chi2_ref = O.chi2(ref, r32(re), r32(im), r32(w))
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")  # noqa: E731
    ctx = Context(0)
    gi, gu, gv = dev(img), dev(u), dev(v)
    vis = ctx.sample_image(gi, dxy, gu, gv, dRA, dDec, PA, pb_fwhm=fwhm).double().cpu().numpy()
    V = vis[:, 0] + 1j * vis[:, 1]
    assert np.max(np.abs(V - ref)) / np.max(np.abs(ref)) <= TOL_VIS
    obs = ctx.register(gu, gv, dev(re), dev(im), dev(w))
    single = ctx.chi2_image(gi, dxy, obs, dRA, dDec, PA, pb_fwhm=fwhm).item()
    assert abs(single - chi2_ref) <= TOL_CHI2 * chi2_ref, (single, chi2_ref)
    batch = ctx.chi2_batch([Request(obs, image=gi, dxy=dxy, dRA=dRA, dDec=dDec, PA=PA,
                                    pb_fwhm=fwhm)] * 2)
    assert batch.cpu().numpy().tolist() == [single] * 2
    ctx.check()
    obs.close()
    ctx.close()
