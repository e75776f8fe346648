"""The allocation-free chi2 entry point against the regular one (GPU).

gal_chi2_image_noalloc_f32 serves callers that may not allocate device
memory (their host application owns it, or an allocation's implicit
synchronisation is not acceptable); it keeps its scratch in a fixed array
inside the library.  It must return what the context-based chi2_image
returns, call after call, although every call reuses the array the previous
one left behind.  This file is collected last on purpose.
"""
import ctypes as ct

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_noalloc_matches_regular_entry_point_twice():
    from paper_1709_06999_gb300 import Context, _native, synth

    lib = _native.load()
    ctx = Context(0)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")  # noqa: E731
    p = synth.small_image_problem(nxy=512, M=20011, seed=21)
    img = dev(p.image)
    u, v, w = dev(p.u), dev(p.v), dev(p.w)
    re = dev(p.noise_re + 0.2)
    im = dev(p.noise_im - 0.1)
    obs = ctx.register(u, v, re, im, w)
    ref = ctx.chi2_image(img, p.dxy, obs, p.dRA, p.dDec, 0.6).item()

    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        out = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.gal_chi2_image_noalloc_f32(img.data_ptr(), 512, p.dxy, p.dRA, p.dDec, 0.6,
                                            u.data_ptr(), v.data_ptr(), re.data_ptr(),
                                            im.data_ptr(), w.data_ptr(), u.numel(),
                                            out.data_ptr(), ct.c_void_p(stream))
        assert st == 0, lib.gal_strerror(st)
        got = out.item()
        assert abs(got - ref) <= 1e-6 * abs(ref), (call, got, ref)


def test_noalloc_rejects_images_beyond_its_scratch():
    from paper_1709_06999_gb300 import _native

    lib = _native.load()
    img = torch.zeros(2048, 2048, dtype=torch.float32, device="cuda")
    x = torch.zeros(8, dtype=torch.float32, device="cuda")
    out = torch.zeros((), dtype=torch.float64, device="cuda")
    st = lib.gal_chi2_image_noalloc_f32(img.data_ptr(), 2048, 1e-8, 0.0, 0.0, 0.0, x.data_ptr(),
                                        x.data_ptr(), x.data_ptr(), x.data_ptr(), x.data_ptr(), 8,
                                        out.data_ptr(), None)
    assert st == -1
