"""FFT plans: the radix of the row and column passes of small float32 sides.

Both radices compute the same discrete Fourier transform (Sect. 4) and must
match the FP64 oracle within the float32 gate; each plan is shared by single
calls and batches, which therefore stay bitwise equal under any plan.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL_VIS = 1e-5
PLANS = [(16, 16), (8, 8), (16, 8), (8, 16)]


def dev(a, dt=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def r32(a):
    return np.asarray(a, np.float32).astype(np.float64)


@pytest.fixture
def restore_plans():
    from paper_1709_06999_gb300 import get_fft_radix, set_fft_radix
    sides = (64, 256, 512)
    saved = {n: get_fft_radix(0, torch.float32, n) for n in sides}
    yield
    for n, (r, c) in saved.items():
        if r:
            set_fft_radix(0, torch.float32, n, r, c)


@pytest.mark.parametrize("nxy", [64, 256, 512])
def test_every_plan_matches_the_oracle(nxy, restore_plans):
    from paper_1709_06999_gb300 import Context, Request, set_fft_radix, get_fft_radix, synth
    ctx = Context(0)
    p = synth.small_image_problem(nxy=nxy, M=20011, seed=nxy)
    ref = O.sample_image(r32(p.image), p.dxy, r32(p.u), r32(p.v), p.dRA, p.dDec, p.PA)
    img, u, v = dev(p.image), dev(p.u), dev(p.v)
    obs = ctx.register(u, v, dev(p.noise_re), dev(p.noise_im), dev(p.w))
    chi2_ref = O.chi2(ref, r32(p.noise_re), r32(p.noise_im), r32(p.w))
    got_plans = {}
    for plan in PLANS:
        set_fft_radix(0, torch.float32, nxy, *plan)
        assert get_fft_radix(0, torch.float32, nxy) == plan
        vis = ctx.sample_image(img, p.dxy, u, v, p.dRA, p.dDec, p.PA).double().cpu().numpy()
        V = vis[:, 0] + 1j * vis[:, 1]
        assert np.max(np.abs(V - ref)) <= TOL_VIS * np.max(np.abs(ref)), plan
        single = ctx.chi2_image(img, p.dxy, obs, p.dRA, p.dDec, p.PA).item()
        assert abs(single - chi2_ref) <= 1e-6 * chi2_ref, plan
        batch = ctx.chi2_batch([Request(obs, image=img, dxy=p.dxy, dRA=p.dRA, dDec=p.dDec,
                                        PA=p.PA)] * 3).cpu().numpy()
        assert batch.tolist() == [single] * 3, plan
        got_plans[plan] = V
    # the two radices round differently but agree far inside the gate
    a, b = got_plans[(16, 16)], got_plans[(8, 8)]
    assert np.max(np.abs(a - b)) <= 1e-6 * np.max(np.abs(ref))
    ctx.check()
    ctx.close()


def test_first_use_fixes_a_plan_and_sides_without_a_choice():
    from paper_1709_06999_gb300 import Context, get_fft_radix, synth
    ctx = Context(0)
    p = synth.small_image_problem(nxy=128, M=5003, seed=3)
    ctx.sample_image(dev(p.image), p.dxy, dev(p.u), dev(p.v), p.dRA, p.dDec, p.PA)
    r, c = get_fft_radix(0, torch.float32, 128)
    assert r in (8, 16) and c in (8, 16)             # fixed at first use (timed)
    assert get_fft_radix(0, torch.float32, 1024) == (16, 16)   # one radix only
    assert get_fft_radix(0, torch.float64, 256) == (8, 8)
    ctx.close()
