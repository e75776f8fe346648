"""Serving loop (gal_server_*): continuous admission, HBM budget, results
identical alone and in a mix of concurrent requests."""
import time

import numpy as np
import pytest
import torch

from paper_1709_06999_gb300 import Context, GalError, Request, Server, synth

pytestmark = pytest.mark.gpu


def dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def datasets(srv, n, dt, seed=0, m_lo=1_000, m_hi=60_000):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        m = int(np.exp(rng.uniform(np.log(m_lo), np.log(m_hi))))
        u, v = synth.uv_loguniform(m, 1e4, 3e6, rng)
        w = synth.weights_uniform(m, rng)
        nre, nim = synth.noise(w, rng)
        out.append(srv.add_data(dev(u, dt), dev(v, dt), dev(nre, dt), dev(nim, dt), dev(w, dt)))
    return out


def requests(data, dt, n, seed=1, sizes=(32, 64, 128, 256, 512)):
    rng = np.random.default_rng(seed)
    ARC = synth.ARCSEC
    imgs = {s: dev(synth.gaussian_image(s, 5.12 * ARC / s, 1.0, 0.3 * ARC, 0.2 * ARC, 0.4), dt)
            for s in sizes}
    prof = {}
    out = []
    for _ in range(n):
        d = data[rng.integers(len(data))]
        s = int(sizes[rng.integers(len(sizes))])
        geo = dict(dRA=rng.uniform(-0.1, 0.1) * ARC, dDec=rng.uniform(-0.1, 0.1) * ARC,
                   PA=rng.uniform(0, np.pi))
        if rng.random() < 0.5:
            out.append(Request(d, image=imgs[s], dxy=5.12 * ARC / s, **geo))
        else:
            nr = 256
            dR = 5.0 * ARC / nr
            key = (s, nr)
            if key not in prof:
                prof[key] = dev(synth.ring_profile(nr, dR, dR / 2), dt)
            out.append(Request(d, intensity=prof[key], nxy=s, dxy=5.12 * ARC / s, Rmin=dR / 2,
                               dR=dR, inc=rng.uniform(0, 1.2), **geo))
    return out


def single(ctx, r):
    obs = ctx.register(*r.obs._tensors)
    kw = dict(pb_fwhm=r.pb_fwhm, full_plane=r.full_plane)
    if r.image is not None:
        return ctx.chi2_image(r.image, r.dxy, obs, r.dRA, r.dDec, r.PA, **kw).item()
    return ctx.chi2_profile(r.intensity, r.Rmin, r.dR, r.nxy, r.dxy, obs, r.inc, r.dRA, r.dDec,
                            r.PA, **kw).item()


@pytest.mark.parametrize("dt", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_alone_equals_mix(dt):
    srv = Server(0, hbm_budget=8 * 10**9, slots=4, max_batch=8)
    data = datasets(srv, 6, dt)
    reqs = requests(data, dt, 48)
    alone = []
    for r in reqs:
        alone.append(srv.wait(srv.submit(r))[0])
    tickets = srv.submit_many(reqs)                   # a burst: slots fill, batches form
    mix = [srv.wait(t)[0] for t in tickets]
    assert mix == alone                               # bitwise
    ctx = Context(0)
    ref = [single(ctx, r) for r in reqs]
    assert ref == alone
    st = srv.stats()
    assert st["completed"] == 2 * len(reqs)
    assert st["launches"] < 2 * len(reqs)            # some requests were batched
    assert st["max_inflight"] > 1                     # and overlapped on the device
    srv.close()


@pytest.mark.parametrize("dt", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_z_order_data(dt):
    """An observation added in Z-order: served alone and in a burst bitwise
    equal, bitwise equal to single calls on a Z-order registration of the
    same arrays, and equal up to summation rounding to the input order."""
    srv = Server(0, hbm_budget=8 * 10**9, slots=4, max_batch=8)
    rng = np.random.default_rng(5)
    m = 40_001
    u, v = synth.uv_loguniform(m, 1e4, 3e6, rng)
    w = synth.weights_uniform(m, rng)
    nre, nim = synth.noise(w, rng)
    arrs = [dev(a, dt) for a in (u, v, nre, nim, w)]
    plain = srv.add_data(*arrs)
    zo = srv.add_data(*arrs, z_order=True)
    reqs_p = requests([plain], dt, 12, seed=3)
    reqs_z = requests([zo], dt, 12, seed=3)   # the same geometries and models
    alone = [srv.wait(srv.submit(r))[0] for r in reqs_z]
    mix = [srv.wait(t)[0] for t in srv.submit_many(reqs_z)]
    assert mix == alone
    ctx = Context(0)
    obs = ctx.register(*arrs, z_order=True)
    single_z = []
    for r in reqs_z:
        if r.image is not None:
            single_z.append(ctx.chi2_image(r.image, r.dxy, obs, r.dRA, r.dDec, r.PA).item())
        else:
            single_z.append(ctx.chi2_profile(r.intensity, r.Rmin, r.dR, r.nxy, r.dxy, obs, r.inc,
                                             r.dRA, r.dDec, r.PA).item())
    assert single_z == alone
    tol = 1e-6 if dt == torch.float32 else 1e-12
    in_order = [srv.wait(srv.submit(r))[0] for r in reqs_p]
    for a, b in zip(alone, in_order):
        assert abs(a - b) <= tol * abs(b)
    srv.close()


def test_beams_alone_equal_mix():
    """Requests with per-request primary beams and some on the full-plane
    spectrum, served alone and in a burst: bitwise equal to each other and to
    single calls."""
    dt = torch.float32
    srv = Server(0, hbm_budget=8 * 10**9, slots=4, max_batch=8)
    data = datasets(srv, 4, dt, seed=8)
    reqs = []
    for k, r in enumerate(requests(data, dt, 24, seed=9)):
        r.pb_fwhm = 0.0 if k % 4 == 3 else (0.4 + 0.02 * k) * r.nxy * r.dxy
        r.full_plane = k % 3 == 1
        reqs.append(r)
    alone = [srv.wait(srv.submit(r))[0] for r in reqs]
    tickets = srv.submit_many(reqs)
    mix = [srv.wait(t)[0] for t in tickets]
    assert mix == alone
    ctx = Context(0)
    assert [single(ctx, r) for r in reqs] == alone
    srv.close()


def test_mixed_precisions_in_one_server():
    srv = Server(0, hbm_budget=8 * 10**9, slots=3, max_batch=4)
    d32 = datasets(srv, 2, torch.float32, seed=3)
    d64 = datasets(srv, 2, torch.float64, seed=4)
    reqs = requests(d32, torch.float32, 10, seed=5) + requests(d64, torch.float64, 10, seed=6)
    order = np.random.default_rng(7).permutation(len(reqs))
    reqs = [reqs[i] for i in order]
    tickets = [srv.submit(r) for r in reqs]
    got = [srv.wait(t)[0] for t in tickets]
    ctx = Context(0)
    assert got == [single(ctx, r) for r in reqs]
    srv.close()


def test_budget_admission_and_rejection():
    dt = torch.float32
    spec512 = 512 * 257 * 8
    # room for the data and about two requests' workspace at a time
    srv0 = Server(0, hbm_budget=10**9, slots=1, max_batch=1)
    probe = datasets(srv0, 1, dt, seed=8, m_lo=20_000, m_hi=20_001)
    data_bytes = srv0.stats()["data_bytes"]
    srv0.close()
    budget = data_bytes + 2 * 3 * spec512 + 4 * 10**6
    srv = Server(0, hbm_budget=budget, slots=4, max_batch=4)
    data = datasets(srv, 1, dt, seed=8, m_lo=20_000, m_hi=20_001)
    reqs = requests(data, dt, 24, seed=9, sizes=(512,))
    tickets = [srv.submit(r) for r in reqs]
    got = [srv.wait(t)[0] for t in tickets]
    ctx = Context(0)
    assert got == [single(ctx, r) for r in reqs]
    st = srv.stats()
    assert st["peak_bytes"] <= budget
    # a request whose workspace can never fit fails alone; the server lives on
    big = Request(data[0], image=dev(np.zeros((4096, 4096)), dt), dxy=1e-8)
    with pytest.raises(GalError):
        srv.wait(srv.submit(big))
    assert srv.wait(srv.submit(reqs[0]))[0] == got[0]
    srv.close()
    del probe


def test_poisson_arrivals_report_latency():
    dt = torch.float32
    srv = Server(0, hbm_budget=8 * 10**9, slots=4, max_batch=8)
    data = datasets(srv, 8, dt, seed=10)
    reqs = requests(data, dt, 300, seed=11)
    rng = np.random.default_rng(12)
    gaps = rng.exponential(1.0 / 2000.0, len(reqs))
    t = time.perf_counter()
    tickets = []
    for r, g in zip(reqs, gaps):
        t += g
        while time.perf_counter() < t:
            pass
        tickets.append(srv.submit(r))
    lat = np.array([srv.wait(tk)[1] for tk in tickets])
    assert np.all(lat > 0) and np.percentile(lat, 50) < 0.05
    srv.close()


def test_submit_rejects_bad_requests():
    srv = Server(0, hbm_budget=10**9, slots=1, max_batch=1)
    data = datasets(srv, 1, torch.float32, seed=13)
    img = dev(np.zeros((48, 48)), torch.float32)               # not a power of two
    with pytest.raises(GalError):
        srv.submit(Request(data[0], image=img, dxy=1e-8))
    img64 = dev(np.zeros((64, 64)), torch.float32)
    for bad in (-1.0, float("nan")):                            # a beam must be >= 0, finite
        with pytest.raises(GalError):
            srv.submit(Request(data[0], image=img64, dxy=1e-8, pb_fwhm=bad))
    with pytest.raises(GalError):
        srv.wait(123456789)                                   # unknown ticket
    srv.close()
