"""Batched chi-square (gal_chi2_batch) and its CUDA-graph form.

Every batched result must be bitwise equal to the single call of the same
request on the same context (same kernels, block partitions and reduction
trees); a few are also checked against the FP64 oracle.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1709_06999_gb300 import Context, GalError, Request, synth

pytestmark = pytest.mark.gpu

TOL_CHI2 = {torch.float64: 1e-12, torch.float32: 1e-6}


def dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def make_obs(ctx, u, v, w, nre, nim, dt):
    # observed = noise only: the chi-square then sums model power plus noise
    return ctx.register(dev(u, dt), dev(v, dt), dev(nre, dt), dev(nim, dt), dev(w, dt))


def single(ctx, r: Request):
    kw = dict(pb_fwhm=r.pb_fwhm, full_plane=r.full_plane)
    if r.image is not None:
        return ctx.chi2_image(r.image, r.dxy, r.obs, r.dRA, r.dDec, r.PA, **kw)
    return ctx.chi2_profile(r.intensity, r.Rmin, r.dR, r.nxy, r.dxy, r.obs, r.inc, r.dRA, r.dDec,
                            r.PA, **kw)


def clone(r: Request, **kw):
    """The same request with some fields replaced."""
    f = dict(image=r.image, intensity=r.intensity, nxy=r.nxy, dxy=r.dxy, dRA=r.dRA, dDec=r.dDec,
             PA=r.PA, Rmin=r.Rmin, dR=r.dR, inc=r.inc, pb_fwhm=r.pb_fwhm,
             full_plane=r.full_plane)
    f.update(kw)
    return Request(r.obs, **f)


def with_beams(reqs):
    """The same requests with a primary beam on two of every three, its width
    varying from request to request like a cube's channels (FWHM ~ lambda)."""
    out = []
    for k, r in enumerate(reqs):
        pb = 0.0 if k % 3 == 2 else (0.3 + 0.04 * k) * r.nxy * r.dxy
        out.append(Request(r.obs, image=r.image, intensity=r.intensity, nxy=r.nxy, dxy=r.dxy,
                           dRA=r.dRA, dDec=r.dDec, PA=r.PA, Rmin=r.Rmin, dR=r.dR, inc=r.inc,
                           pb_fwhm=pb))
    return out


def mixed_requests(ctx, dt, seed=0, n_img=10, n_prof=6):
    """Cube channels of several sides plus profile walkers sharing one dataset."""
    rng = np.random.default_rng(seed)
    cube = synth.spectral_cube(n_chan=n_img, sizes=(32, 64, 128, 256), m_lo=2_000, m_hi=30_000,
                               seed=seed)
    reqs, keep = [], []
    for ch in cube:
        obs = make_obs(ctx, ch.u, ch.v, ch.w, ch.noise_re, ch.noise_im, dt)
        img = dev(ch.image, dt)
        keep.append((obs, img))
        reqs.append(Request(obs, image=img, dxy=ch.dxy, dRA=ch.dRA, dDec=ch.dDec, PA=ch.PA))
    q = synth.profile_problem(nxy=128, M=20_000, nr=512, seed=seed + 1, dxy=0.04 * synth.ARCSEC)
    obs = make_obs(ctx, q.u, q.v, q.w, q.noise_re, q.noise_im, dt)
    keep.append(obs)
    for p in synth.walker_params(n_prof, seed=seed + 2):
        I = dev(synth.ring_profile(512, q.dR, q.Rmin, p["r0"], p["width"], p["power"]), dt)
        keep.append(I)
        reqs.append(Request(obs, intensity=I, nxy=q.nxy, dxy=q.dxy, Rmin=q.Rmin, dR=q.dR,
                            inc=p["inc"], dRA=p["dRA"], dDec=p["dDec"], PA=p["PA"]))
    order = rng.permutation(len(reqs))
    return [reqs[i] for i in order], keep


@pytest.mark.parametrize("dt", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_batch_equals_single_calls_bitwise(dt):
    ctx = Context(0)
    reqs, keep = mixed_requests(ctx, dt)
    got = ctx.chi2_batch(reqs)
    want = torch.stack([single(ctx, r) for r in reqs])
    assert torch.equal(got, want), (got - want).abs().max().item()
    assert all(math.isfinite(x) and x > 0 for x in got.tolist())


def test_batch_matches_oracle():
    ctx = Context(0)
    dt = torch.float32
    reqs, keep = mixed_requests(ctx, dt, seed=5, n_img=3, n_prof=2)
    got = ctx.chi2_batch(reqs).cpu().numpy()
    for r, g in zip(reqs, got):
        o = r.obs
        u, v, re, im, w = (t.double().cpu().numpy() for t in o._tensors)
        if r.image is not None:
            ref = oracle.chi2_image(r.image.double().cpu().numpy(), r.dxy, u, v, re, im, w,
                                    r.dRA, r.dDec, r.PA)
        else:
            ref = oracle.chi2_profile(r.intensity.double().cpu().numpy(), r.Rmin, r.dR, r.nxy,
                                      r.dxy, u, v, re, im, w, r.dRA, r.dDec, r.PA, r.inc)
        assert abs(g - ref) <= TOL_CHI2[dt] * abs(ref), (g, ref)


def test_more_than_one_launch_per_pass_and_odd_members():
    """40 requests of one side (two chunks), an unbatchable side, an empty
    observation and a mix of precisions in one call."""
    ctx = Context(0)
    rng = np.random.default_rng(9)
    reqs, keep = [], []
    p = synth.small_image_problem(nxy=64, M=3_000, seed=9)
    obs32 = make_obs(ctx, p.u, p.v, p.w, p.noise_re, p.noise_im, torch.float32)
    obs64 = make_obs(ctx, p.u, p.v, p.w, p.noise_re, p.noise_im, torch.float64)
    empty = ctx.register(*(torch.empty(0, dtype=torch.float32, device="cuda") for _ in range(5)))
    for k in range(40):
        img = dev(p.image * (1.0 + 0.01 * k), torch.float32)
        keep.append(img)
        reqs.append(Request(obs32, image=img, dxy=p.dxy, dRA=p.dRA, PA=0.1 * k))
    small = dev(p.image[24:40, 24:40], torch.float32)          # nxy = 16: single-call path
    reqs.append(Request(obs32, image=small, dxy=p.dxy))
    reqs.append(Request(empty, image=dev(p.image, torch.float32), dxy=p.dxy))
    img64 = dev(p.image, torch.float64)
    reqs.append(Request(obs64, image=img64, dxy=p.dxy, dDec=p.dDec))
    keep += [small, img64]
    order = rng.permutation(len(reqs))
    reqs = [reqs[i] for i in order]
    got = ctx.chi2_batch(reqs)
    want = torch.stack([single(ctx, r) for r in reqs])
    assert torch.equal(got, want)
    k_empty = [i for i, r in enumerate(reqs) if r.obs is empty][0]
    assert got[k_empty].item() == 0.0


def test_tuning_does_not_change_results():
    ctx = Context(0)
    reqs, keep = mixed_requests(ctx, torch.float32, seed=3, n_img=6, n_prof=3)
    ctx.set_batch_tuning(False)
    a = ctx.chi2_batch(reqs)
    ctx2 = Context(0)
    ctx2.set_batch_tuning(True)
    reqs2 = [Request(ctx2.register(*r.obs._tensors), image=r.image, intensity=r.intensity,
                     nxy=r.nxy, dxy=r.dxy, dRA=r.dRA, dDec=r.dDec, PA=r.PA, Rmin=r.Rmin, dR=r.dR,
                     inc=r.inc) for r in reqs]
    b = ctx2.chi2_batch(reqs2)
    c = ctx2.chi2_batch(reqs2)   # cached shape
    assert torch.equal(a, b) and torch.equal(b, c)


def test_launch_shapes_do_not_change_results():
    """Every launch shape (row-pass blocks per SM, requests per launch,
    gather fold) gives the single calls' results bit for bit, on windows
    staged in shared memory (sides 32..128) and read through L2 (side 256);
    a shape set for a batch key is read back and used."""
    ctx = Context(0)
    reqs, keep = mixed_requests(ctx, torch.float32, seed=11, n_img=12, n_prof=4)
    want = torch.stack([single(ctx, r) for r in reqs])
    n, nmax = len(reqs), max(r.nxy for r in reqs)
    assert ctx.batch_shape(torch.float32, n, nmax) == ((1, 32, 4), False)  # the default
    for shape in [(1, 32, 1), (2, 8, 2), (4, 16, 8), (1, 3, 4), (8, 1, 8), (2, 32, 3)]:
        ctx.set_batch_shape(torch.float32, n, nmax, *shape)
        assert ctx.batch_shape(torch.float32, n, nmax) == (shape, True)
        got = ctx.chi2_batch(reqs)
        assert torch.equal(got, want), shape


def test_tuner_keeps_a_candidate_shape():
    ctx = Context(0)
    reqs, keep = mixed_requests(ctx, torch.float64, seed=13, n_img=5, n_prof=3)
    n, nmax = len(reqs), max(r.nxy for r in reqs)
    got = ctx.chi2_batch(reqs)                        # tunes this key
    (rb, jobs, fold), kept = ctx.batch_shape(torch.float64, n, nmax)
    assert kept
    assert (rb, jobs) in {(1, 32), (2, 32), (4, 32), (1, 8), (2, 8), (4, 16)}
    assert fold in (1, 2, 4, 8)
    assert ctx.batch_shape(torch.float32, n, nmax)[1] is False   # other precision untouched
    assert torch.equal(got, torch.stack([single(ctx, r) for r in reqs]))


def test_batch_shape_validation():
    ctx = Context(0)
    for bad in ((torch.float32, 0, 256, 1, 32, 4), (torch.float32, 4, 300, 1, 32, 4),
                (torch.float32, 4, 256, 0, 32, 4), (torch.float32, 4, 256, 9, 32, 4),
                (torch.float32, 4, 256, 1, 33, 4), (torch.float32, 4, 256, 1, 0, 4),
                (torch.float32, 4, 256, 1, 32, 0), (torch.float32, 4, 256, 1, 32, 9)):
        with pytest.raises(GalError):
            ctx.set_batch_shape(*bad)
    with pytest.raises(ValueError):
        ctx.set_batch_shape(torch.int32, 4, 256, 1, 32, 4)


def test_graph_replay_update_and_regrowth():
    ctx = Context(0)
    reqs, keep = mixed_requests(ctx, torch.float32, seed=7, n_img=5, n_prof=3)
    g = ctx.capture_batch(reqs)
    want = torch.stack([single(ctx, r) for r in reqs])
    out = g.launch().clone()
    torch.cuda.synchronize()
    assert torch.equal(out, want)
    # rewrite one image and one profile in place: the replay sees the new values
    ki = next(i for i, r in enumerate(reqs) if r.image is not None)
    kp = next(i for i, r in enumerate(reqs) if r.intensity is not None)
    reqs[ki].image.mul_(0.5)
    reqs[kp].intensity.mul_(2.0)
    out = g.launch().clone()
    want = torch.stack([single(ctx, r) for r in reqs])
    assert torch.equal(out, want)
    # new scalars, same structure: update in place
    new = [Request(r.obs, image=r.image, intensity=r.intensity, nxy=r.nxy, dxy=r.dxy,
                   dRA=r.dRA + 1e-7, dDec=r.dDec, PA=r.PA + 0.3, Rmin=r.Rmin, dR=r.dR, inc=r.inc)
           for r in reqs]
    g.update(new)
    out = g.launch().clone()
    want = torch.stack([single(ctx, r) for r in new])
    assert torch.equal(out, want)
    # a bigger batch reallocates the workspace; the graph re-records itself
    big, keep2 = mixed_requests(ctx, torch.float32, seed=8, n_img=12, n_prof=4)
    ctx.chi2_batch(big)
    out = g.launch().clone()
    assert torch.equal(out, want)
    # a different structure is refused
    with pytest.raises(GalError):
        g.update(new[:-1])
    g.close()


def test_invalid_request_launches_nothing():
    ctx = Context(0)
    reqs, keep = mixed_requests(ctx, torch.float32, seed=11, n_img=2, n_prof=1)
    n0 = ctx.launch_count()
    bad = list(reqs) + [Request(reqs[0].obs, image=reqs[0].image, dxy=-1.0)]
    with pytest.raises(GalError):
        ctx.chi2_batch(bad)
    assert ctx.launch_count() == n0
    out = ctx.chi2_batch([])
    assert out.numel() == 0


def test_cube_channels_at_their_sizes_match_oracle():
    """Keplerian cube channels at the cube's image sides (512-2048) and
    observation sizes (1e5-2e5 points) through one batch, against the oracle."""
    ctx = Context(0)
    dt = torch.float32
    cube = synth.spectral_cube(n_chan=6, sizes=(512, 1024, 2048), m_lo=100_000, m_hi=200_000,
                               seed=21)
    reqs, keep = [], []
    for ch in cube:
        obs = make_obs(ctx, ch.u, ch.v, ch.w, ch.noise_re, ch.noise_im, dt)
        img = dev(ch.image, dt)
        keep.append((obs, img))
        reqs.append(Request(obs, image=img, dxy=ch.dxy, dRA=ch.dRA, dDec=ch.dDec, PA=ch.PA))
    assert {r.nxy for r in reqs} == {512, 1024, 2048}
    got = ctx.chi2_batch(reqs).cpu().numpy()
    for r, g in zip(reqs, got):
        u, v, re, im, w = (t.double().cpu().numpy() for t in r.obs._tensors)
        ref = oracle.chi2_image(r.image.double().cpu().numpy(), r.dxy, u, v, re, im, w, r.dRA,
                                r.dDec, r.PA)
        assert abs(g - ref) <= TOL_CHI2[dt] * abs(ref), (r.nxy, g, ref)


@pytest.mark.parametrize("dt", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_batch_with_beams_equals_single_calls_bitwise(dt):
    """Per-request primary beams (images and profiles, with and without a
    beam in one batch): bitwise the single calls with the same beam."""
    ctx = Context(0)
    reqs, keep = mixed_requests(ctx, dt, seed=13, n_img=8, n_prof=5)
    reqs = with_beams(reqs)
    got = ctx.chi2_batch(reqs)
    want = torch.stack([single(ctx, r) for r in reqs])
    assert torch.equal(got, want), (got - want).abs().max().item()
    plain = ctx.chi2_batch([Request(r.obs, image=r.image, intensity=r.intensity, nxy=r.nxy,
                                    dxy=r.dxy, dRA=r.dRA, dDec=r.dDec, PA=r.PA, Rmin=r.Rmin,
                                    dR=r.dR, inc=r.inc) for r in reqs])
    # without a beam the result is the plain batch's; with one it differs for the
    # cube channels (about 1 Jy each; the test profiles are ~1e-14 Jy per pixel,
    # far below the unit noise, so no factor can move their chi-square)
    for k, r in enumerate(reqs):
        if r.pb_fwhm == 0.0:
            assert got[k].item() == plain[k].item(), k
        elif r.image is not None:
            assert got[k].item() != plain[k].item(), k


def test_batch_with_beams_matches_oracle():
    ctx = Context(0)
    dt = torch.float32
    reqs, keep = mixed_requests(ctx, dt, seed=15, n_img=3, n_prof=2)
    reqs = with_beams(reqs)
    got = ctx.chi2_batch(reqs).cpu().numpy()
    for r, g in zip(reqs, got):
        u, v, re, im, w = (t.double().cpu().numpy() for t in r.obs._tensors)
        if r.image is not None:
            ref = oracle.chi2_image(r.image.double().cpu().numpy(), r.dxy, u, v, re, im, w,
                                    r.dRA, r.dDec, r.PA, pb_fwhm=r.pb_fwhm)
        else:
            ref = oracle.chi2_profile(r.intensity.double().cpu().numpy(), r.Rmin, r.dR, r.nxy,
                                      r.dxy, u, v, re, im, w, r.dRA, r.dDec, r.PA, r.inc,
                                      pb_fwhm=r.pb_fwhm)
        assert abs(g - ref) <= TOL_CHI2[dt] * abs(ref), (g, ref, r.pb_fwhm)


def test_graph_with_beams_replay_and_update():
    """A captured batch with beams replays to the single calls' results; new
    offsets and position angles (which move each beam's centre on the grid)
    update it in place; adding or removing a beam changes its structure."""
    ctx = Context(0)
    reqs, keep = mixed_requests(ctx, torch.float32, seed=17, n_img=5, n_prof=3)
    reqs = with_beams(reqs)
    g = ctx.capture_batch(reqs)
    out = g.launch().clone()
    assert torch.equal(out, torch.stack([single(ctx, r) for r in reqs]))
    new = [Request(r.obs, image=r.image, intensity=r.intensity, nxy=r.nxy, dxy=r.dxy,
                   dRA=r.dRA + 2e-7, dDec=r.dDec - 1e-7, PA=r.PA + 0.4, Rmin=r.Rmin, dR=r.dR,
                   inc=r.inc, pb_fwhm=r.pb_fwhm * 1.1) for r in reqs]
    g.update(new)
    out = g.launch().clone()
    assert torch.equal(out, torch.stack([single(ctx, r) for r in new]))
    flipped = list(new)
    k = next(i for i, r in enumerate(new) if r.pb_fwhm == 0.0)
    r = new[k]
    flipped[k] = Request(r.obs, image=r.image, intensity=r.intensity, nxy=r.nxy, dxy=r.dxy,
                         dRA=r.dRA, dDec=r.dDec, PA=r.PA, Rmin=r.Rmin, dR=r.dR, inc=r.inc,
                         pb_fwhm=0.5 * r.nxy * r.dxy)
    with pytest.raises(GalError):
        g.update(flipped)
    g.close()


def test_invalid_beam_in_batch_launches_nothing():
    ctx = Context(0)
    reqs, keep = mixed_requests(ctx, torch.float32, seed=19, n_img=2, n_prof=1)
    n0 = ctx.launch_count()
    r = reqs[0]
    for bad in (-1.0, float("nan")):
        with pytest.raises(GalError):
            ctx.chi2_batch(list(reqs) + [Request(r.obs, image=r.image, intensity=r.intensity,
                                                 nxy=r.nxy, dxy=r.dxy, pb_fwhm=bad)])
    assert ctx.launch_count() == n0


@pytest.mark.parametrize("dt", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_batch_full_plane_equals_single_calls_bitwise(dt):
    """Full-plane requests (every other one, some with a beam) batched with
    half-plane ones: bitwise the single calls with the same options."""
    ctx = Context(0)
    reqs, keep = mixed_requests(ctx, dt, seed=23, n_img=8, n_prof=5)
    reqs = [clone(r, full_plane=(k % 2 == 0),
                  pb_fwhm=0.0 if k % 3 == 2 else (0.35 + 0.03 * k) * r.nxy * r.dxy)
            for k, r in enumerate(reqs)]
    got = ctx.chi2_batch(reqs)
    want = torch.stack([single(ctx, r) for r in reqs])
    assert torch.equal(got, want), (got - want).abs().max().item()
    # and within rounding of the half-plane results (the C2C/R2C check) where
    # every point lies inside the grid: beyond it the two paths clamp to
    # different node ranges (-N/2..N/2-1 against 0..N/2 with the fold)
    half = ctx.chi2_batch([clone(r, full_plane=False) for r in reqs])
    inside = 0
    for k, r in enumerate(reqs):
        u, v = (t.double() for t in r.obs._tensors[:2])
        rho = torch.sqrt(torch.max(u * u + v * v)).item()
        if rho * r.nxy * r.dxy < r.nxy / 2 - 1:
            inside += 1
            rel = abs(got[k].item() - half[k].item()) / abs(half[k].item())
            assert rel <= 2 * TOL_CHI2[dt], (k, rel)
    assert inside >= 3


def test_batch_full_plane_matches_oracle():
    ctx = Context(0)
    dt = torch.float32
    reqs, keep = mixed_requests(ctx, dt, seed=25, n_img=3, n_prof=2)
    reqs = [clone(r, full_plane=True, pb_fwhm=0.5 * r.nxy * r.dxy if k % 2 else 0.0)
            for k, r in enumerate(reqs)]
    got = ctx.chi2_batch(reqs).cpu().numpy()
    for r, g in zip(reqs, got):
        u, v, re, im, w = (t.double().cpu().numpy() for t in r.obs._tensors)
        kw = dict(pb_fwhm=r.pb_fwhm, full_plane=True)
        if r.image is not None:
            ref = oracle.chi2_image(r.image.double().cpu().numpy(), r.dxy, u, v, re, im, w,
                                    r.dRA, r.dDec, r.PA, **kw)
        else:
            ref = oracle.chi2_profile(r.intensity.double().cpu().numpy(), r.Rmin, r.dR, r.nxy,
                                      r.dxy, u, v, re, im, w, r.dRA, r.dDec, r.PA, r.inc, **kw)
        assert abs(g - ref) <= TOL_CHI2[dt] * abs(ref), (g, ref)


def test_graph_full_plane_replay_update_and_structure():
    ctx = Context(0)
    reqs, keep = mixed_requests(ctx, torch.float32, seed=27, n_img=4, n_prof=2)
    reqs = [clone(r, full_plane=(k % 2 == 1)) for k, r in enumerate(reqs)]
    g = ctx.capture_batch(reqs)
    out = g.launch().clone()
    assert torch.equal(out, torch.stack([single(ctx, r) for r in reqs]))
    new = [clone(r, PA=r.PA + 0.7, dRA=r.dRA - 1e-7) for r in reqs]
    g.update(new)
    out = g.launch().clone()
    assert torch.equal(out, torch.stack([single(ctx, r) for r in new]))
    with pytest.raises(GalError):  # switching a request's spectrum path changes the structure
        g.update([clone(new[0], full_plane=not new[0].full_plane)] + new[1:])
    g.close()


def test_invalid_full_plane_in_batch_launches_nothing():
    ctx = Context(0)
    reqs, keep = mixed_requests(ctx, torch.float32, seed=29, n_img=2, n_prof=1)
    n0 = ctx.launch_count()
    r = next(r for r in reqs if r.image is not None)
    small = torch.zeros((8, 8), dtype=torch.float32, device="cuda")  # below the f32 full-plane range
    with pytest.raises(GalError):
        ctx.chi2_batch(list(reqs) + [Request(r.obs, image=small, dxy=r.dxy, full_plane=True)])
    assert ctx.launch_count() == n0
