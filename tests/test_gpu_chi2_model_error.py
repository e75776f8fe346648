"""The chi-square kernels measured on the model error itself.

With observed data equal to a model, Eq. chap6.eq:def.chi.square reduces to
sum_k w_k |V_k - V_model,k|^2: the weighted squared difference of the two
visibility sets, with no noise term to hide it.  So:

* observed = the library's own sample_image output gives chi2 == 0 exactly,
  which holds only if the chi-square-only gather variant computes bit for bit
  the visibilities of the sampling variant (same window, same cells, same
  phase), on the full-size workload: 4096^2 image, 5e6 uv points, pruned
  window staged in shared memory;
* observed = the FP64 oracle's model gives a chi2 bounded by
  sum_k w_k (tol max|V|)^2, with tol the visibility gate of the path (1e-5
  normwise for float32, 1e-12 for float64).  A model error of relative size
  delta moves this chi2 by about delta^2 sum w |V|^2, so the check is as tight
  as the visibility gate itself (a noise-dominated chi2 is not).

Cases: the large image (nxy 4096, M 5e6, float32 bulk with the float64
reduction, and the float64 path), the profile case (nxy 1024, M 1e6, nr 8192)
and requests of a batched spectral cube.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL_VIS = {torch.float64: 1e-12, torch.float32: 1e-5}
DTYPES = [torch.float64, torch.float32]
IDS = ["f64", "f32"]


def dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def rounded(a, dt):
    return np.asarray(a, dtype=np.float32 if dt == torch.float32 else np.float64).astype(np.float64)


def bound(model, w, dt):
    """sum_k w_k (tol max|V|)^2 for observed data equal to the oracle model,
    plus the rounding of that model to the path's precision (at most half an
    ulp per component)."""
    vmax = float(np.max(np.abs(model)))
    eps = 2.0 ** -24 if dt == torch.float32 else 2.0 ** -53
    per = TOL_VIS[dt] * vmax + 2.0 * eps * vmax
    return float(np.sum(w)) * per * per


@pytest.fixture(scope="module")
def ctx():
    from paper_1709_06999_gb300 import Context
    c = Context(0)
    yield c
    c.check()
    c.close()


@pytest.fixture(scope="module")
def large():
    from paper_1709_06999_gb300 import synth
    return synth.large_image_problem()


@pytest.fixture(scope="module")
def large_models(large):
    """Oracle model of the large case on the inputs each path sees."""
    p = large
    out = {}
    for dt in DTYPES:
        R = lambda a: rounded(a, dt)  # noqa: E731
        G = O.half_spectrum(R(p.image))
        out[dt] = O.sample_spectrum(G, p.image.shape[0], p.dxy, R(p.u), R(p.v), p.dRA, p.dDec,
                                    p.PA)
    return out


@pytest.mark.parametrize("dt", DTYPES, ids=IDS)
def test_large_chi2_zero_at_own_model(ctx, large, dt):
    p = large
    img, u, v, w = dev(p.image, dt), dev(p.u, dt), dev(p.v, dt), dev(p.w, dt)
    vis = ctx.sample_image(img, p.dxy, u, v, p.dRA, p.dDec, p.PA)
    obs = ctx.register(u, v, vis[:, 0].contiguous(), vis[:, 1].contiguous(), w)
    assert ctx.chi2_image(img, p.dxy, obs, p.dRA, p.dDec, p.PA).item() == 0.0
    # the same observation, another position angle: a plain positive chi2
    assert ctx.chi2_image(img, p.dxy, obs, p.dRA, p.dDec, p.PA + 0.3).item() > 0.0


@pytest.mark.parametrize("dt", DTYPES, ids=IDS)
def test_large_chi2_noise_free(ctx, large, large_models, dt):
    p = large
    model = large_models[dt]
    img, u, v = dev(p.image, dt), dev(p.u, dt), dev(p.v, dt)
    obs = ctx.register(u, v, dev(model.real, dt), dev(model.imag, dt), dev(p.w, dt))
    chi2 = ctx.chi2_image(img, p.dxy, obs, p.dRA, p.dDec, p.PA).item()
    lim = bound(model, rounded(p.w, dt), dt)
    assert 0.0 <= chi2 <= lim, (chi2, lim)
    # the check has teeth: an observation 10x the gate (10 tol max|V|) away
    # from the model at every point fails it
    off = model.real + 10.0 * TOL_VIS[dt] * float(np.max(np.abs(model)))
    obs2 = ctx.register(u, v, dev(off, dt), dev(model.imag, dt), dev(p.w, dt))
    assert ctx.chi2_image(img, p.dxy, obs2, p.dRA, p.dDec, p.PA).item() > lim


@pytest.mark.parametrize("dt", DTYPES, ids=IDS)
def test_profile_chi2_noise_free(ctx, dt):
    from paper_1709_06999_gb300 import synth
    q = synth.profile_problem()
    R = lambda a: rounded(a, dt)  # noqa: E731
    model = O.sample_profile(R(q.intensity), q.Rmin, q.dR, q.nxy, q.dxy, R(q.u), R(q.v), q.dRA,
                             q.dDec, q.PA, q.inc)
    I_d, u_d, v_d = dev(q.intensity, dt), dev(q.u, dt), dev(q.v, dt)
    obs = ctx.register(u_d, v_d, dev(model.real, dt), dev(model.imag, dt), dev(q.w, dt))
    chi2 = ctx.chi2_profile(I_d, q.Rmin, q.dR, q.nxy, q.dxy, obs, q.inc, q.dRA, q.dDec,
                            q.PA).item()
    lim = bound(model, R(q.w), dt)
    assert 0.0 <= chi2 <= lim, (chi2, lim)
    vis = ctx.sample_profile(I_d, q.Rmin, q.dR, q.nxy, q.dxy, u_d, v_d, q.inc, q.dRA, q.dDec, q.PA)
    obs0 = ctx.register(u_d, v_d, vis[:, 0].contiguous(), vis[:, 1].contiguous(), dev(q.w, dt))
    assert ctx.chi2_profile(I_d, q.Rmin, q.dR, q.nxy, q.dxy, obs0, q.inc, q.dRA, q.dDec,
                            q.PA).item() == 0.0


@pytest.mark.parametrize("dt", DTYPES, ids=IDS)
def test_batched_cube_noise_free(ctx, dt):
    """Cube channels of each side (512, 1024, 2048) in one gal_chi2_batch:
    observed = oracle model gives chi2 within the bound, observed = the
    library's own samples gives exactly 0, and both equal the single calls."""
    from paper_1709_06999_gb300 import Request, synth
    cube = [ch for k, n in enumerate((512, 1024, 2048))
            for ch in synth.spectral_cube(n_chan=2, sizes=(n,), m_lo=100_000, m_hi=400_000,
                                          seed=17 + k)]
    reqs, lims, keep = [], [], []
    R = lambda a: rounded(a, dt)  # noqa: E731
    for ch in cube:
        model = O.sample_image(R(ch.image), ch.dxy, R(ch.u), R(ch.v), ch.dRA, ch.dDec, ch.PA)
        img, u, v, w = dev(ch.image, dt), dev(ch.u, dt), dev(ch.v, dt), dev(ch.w, dt)
        obs = ctx.register(u, v, dev(model.real, dt), dev(model.imag, dt), w)
        vis = ctx.sample_image(img, ch.dxy, u, v, ch.dRA, ch.dDec, ch.PA)
        obs0 = ctx.register(u, v, vis[:, 0].contiguous(), vis[:, 1].contiguous(), w)
        keep += [obs, obs0, img]
        kw = dict(image=img, dxy=ch.dxy, dRA=ch.dRA, dDec=ch.dDec, PA=ch.PA)
        reqs += [Request(obs, **kw), Request(obs0, **kw)]
        lims.append(bound(model, R(ch.w), dt))
    assert sorted({ch.image.shape[0] for ch in cube}) == [512, 1024, 2048]
    got = ctx.chi2_batch(reqs).cpu().numpy()
    for k, lim in enumerate(lims):
        assert 0.0 <= got[2 * k] <= lim, (k, got[2 * k], lim)
        assert got[2 * k + 1] == 0.0, (k, got[2 * k + 1])
    single = [ctx.chi2_image(r.image, r.dxy, r.obs, r.dRA, r.dDec, r.PA).item() for r in reqs]
    assert got.tolist() == single
