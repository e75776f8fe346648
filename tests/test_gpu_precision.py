"""The error of the index and of the phase arithmetic, each isolated, at all
5e6 points of the large case (nxy 4096, its uv coverage and geometry).

Two images have spectra that every FFT path computes exactly, so that the
visibility error left is the sampling arithmetic's alone:

* a unit point at pixel (0, 0) (offset -N/2, -N/2 from the phase centre):
  its half spectrum is G[r][c] = (-1)^(r + c) exactly in any precision (one
  non-zero input reaches every output through twiddles of 1 and -1 only).
  With no offset the visibility is the bilinear interpolation of that
  checkerboard, (1 - 2 fu)(1 - 2 fv) up to sign, so an error d in a cell
  fraction moves it by about 2 d: the difference to the oracle (FP64 indices
  of the same float32 u, v) measures the uv -> cell index error of Sect. 3.2
  and App. D;
* a unit point at the phase centre: G = 1 everywhere, the visibility is the
  phase factor exp(2 pi i (u dRA + v dDec)) alone (Sect. 3.2, App. D sign).

Bounds (float32 path: float-float index and phase, the reading stated in the
design notes; float64 path: plain FP64):
  index  |dV| <= 2 (d_u + d_v) + lerp rounding; the cell fraction is rounded
         once to float (<= 2^-25) after a float-float position good to
         ~2^-45 |x|, the lerp adds ~4 roundings of values <= 1:  <= 1e-6
         (a plain float32 position of |x| ~ 60 cells would give ~1.5e-5)
  phase  angle: one float rounding of the reduced turns (<= 2^-24 turn) and of
         the product by 2 pi, plus the documented absolute error of CUDA's
         __sincosf on [-pi, pi] (2^-21.41 each for sin and cos):  <= 1.5e-6
  float64: the kernel's fraction is exact to rounding, but the oracle forms
         the row index as N/2 + v'/du in FP64, which rounds at ulp(N/2) =
         2^-41 for N = 4096: index 2e-12 (twice that, doubled by the
         checkerboard); phase 1e-14
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

BOUNDS = {"index": {torch.float32: 1e-6, torch.float64: 2e-12},
          "phase": {torch.float32: 1.5e-6, torch.float64: 1e-14}}


def dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def rounded(a, dt):
    return np.asarray(a, dtype=np.float32 if dt == torch.float32 else np.float64).astype(np.float64)


@pytest.fixture(scope="module")
def case():
    from paper_1709_06999_gb300 import Context, synth
    p = synth.large_image_problem()
    return Context(0), p


@pytest.mark.parametrize("dt", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_index_error_isolated(case, dt):
    ctx, p = case
    N = p.image.shape[0]
    img = np.zeros((N, N))
    img[0, 0] = 1.0
    u, v = rounded(p.u, dt), rounded(p.v, dt)
    ref = O.sample_image(img, p.dxy, u, v, 0.0, 0.0, p.PA)
    got = ctx.sample_image(dev(img, dt), p.dxy, dev(p.u, dt), dev(p.v, dt), 0.0, 0.0,
                           p.PA).double().cpu().numpy()
    err = np.max(np.abs(got[:, 0] + 1j * got[:, 1] - ref))
    assert err <= BOUNDS["index"][dt], err
    # the checkerboard makes the test sensitive: a quarter-cell shift of every
    # point would change the visibilities by about one half
    assert np.max(np.abs(ref)) > 0.99


@pytest.mark.parametrize("dt", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_phase_error_isolated(case, dt):
    ctx, p = case
    N = p.image.shape[0]
    img = np.zeros((N, N))
    img[N // 2, N // 2] = 1.0
    u, v = rounded(p.u, dt), rounded(p.v, dt)
    exact = np.exp(2j * np.pi * (u * p.dRA + v * p.dDec))
    ref = O.sample_image(img, p.dxy, u, v, p.dRA, p.dDec, p.PA)
    assert np.max(np.abs(ref - exact)) <= 1e-12      # the oracle: phase factor alone
    got = ctx.sample_image(dev(img, dt), p.dxy, dev(p.u, dt), dev(p.v, dt), p.dRA, p.dDec,
                           p.PA).double().cpu().numpy()
    err = np.max(np.abs(got[:, 0] + 1j * got[:, 1] - exact))
    assert err <= BOUNDS["phase"][dt], err
