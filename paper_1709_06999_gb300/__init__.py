"""GB300-native (sm_103a) synthetic visibilities and chi-square for radio
interferometry: the hot path of GALARIO (arXiv 1709.06999) as hand-written
CUDA kernels behind a C ABI (include/galario_gb300.h).

    from paper_1709_06999_gb300 import Context
    ctx = Context(0)
    obs = ctx.register(u, v, re, im, w)            # device tensors, float32 or float64
    chi2 = ctx.chi2_image(image, dxy, obs, dRA, dDec, PA)
"""
from .api import (BatchGraph, Context, GalError, Observation, Request, Server,  # noqa: F401
                  chi2_image, chi2_profile, default_context, get_fft_radix, get_image_size,
                  sample_image, sample_profile, set_fft_radix, sweep)
