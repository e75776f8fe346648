"""get_image_size (Sect. 3.3): the oracle against the paper's matrix-size table.

The table (tests/golden/matrix_sizes.txt) gives, per array configuration, the
shortest and longest baselines and the image sizes of criteria (iia) and
(iib), the pixel size and the resolution.  A uv set holding exactly those two
baselines reproduces them.
"""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "matrix_sizes.txt")
ARCSEC = math.pi / 648000.0
WAVELENGTH = {"ALMA": 1.3e-3, "VLA": 7.0e-3}
DISH = {"ALMA": 12.0, "VLA": 25.0}
# Primary-beam FWHM = K lambda / D.  The paper does not state K; every K in
# (1.416, 1.845] reproduces its N_lm (iib) column with these dish sizes (the
# bounds come from ALMA C43-3/C43-8 and VLA A/B), the usual 1.13 does not.
K_BEAM = 1.5


def rows():
    out = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            a, cfg, bmin, bmax, n1, n2, dth, res = line.split()
            out.append((a, cfg, float(bmin), float(bmax), int(n1), int(n2), float(dth),
                        float(res)))
    return out


def uv_of(array, bmin, bmax):
    lam = WAVELENGTH[array]
    # two baselines along different axes, plus a third at 45 degrees in between
    r = np.array([bmin, bmax, 0.5 * (bmin + bmax)]) / lam
    ang = np.array([0.3, 2.0, 4.0])
    return r * np.cos(ang), r * np.sin(ang)


@pytest.mark.parametrize("row", rows(), ids=lambda r: f"{r[0]}-{r[1]}")
def test_table_criterion_iia(row):
    array, cfg, bmin, bmax, n_iia, n_iib, dtheta, res = row
    u, v = uv_of(array, bmin, bmax)
    n, dxy = oracle.image_size(u, v)
    assert n == n_iia
    # the printed pixel sizes are rounded to 0.001"
    assert abs(dxy / ARCSEC - dtheta) <= 0.0005 + 1e-9
    # resolution 1 / rho_max (the table's theta_res), same rounding
    assert abs(WAVELENGTH[array] / bmax / ARCSEC - res) <= 0.0005 + 1e-9


@pytest.mark.parametrize("row", rows(), ids=lambda r: f"{r[0]}-{r[1]}")
def test_table_criterion_iib(row):
    array, cfg, bmin, bmax, n_iia, n_iib, dtheta, res = row
    u, v = uv_of(array, bmin, bmax)
    pb = K_BEAM * WAVELENGTH[array] / DISH[array]
    n, dxy = oracle.image_size(u, v, PB=pb)
    assert n == n_iib
    # the field covers the beam and f_min times the largest recoverable scale
    assert n * dxy >= pb * (1 - 1e-12)


def test_beam_constant_range_is_what_the_table_allows():
    """The (iib) column pins K to (1.416, 1.845]: just outside fails a row."""
    def all_match(k):
        for array, cfg, bmin, bmax, n_iia, n_iib, _, _ in rows():
            u, v = uv_of(array, bmin, bmax)
            if oracle.image_size(u, v, PB=k * WAVELENGTH[array] / DISH[array])[0] != n_iib:
                return False
        return True
    assert all_match(1.42) and all_match(1.84)
    assert not all_match(1.40) and not all_match(1.86) and not all_match(1.13)


def test_power_of_two_boundaries():
    # need exactly a power of two -> that power; just above -> the next one
    lam_ratio = 1024.0 / (2 * 2.5 * 0.6 * 5)   # rho_max / rho_min giving need = 1024
    n, _ = oracle.image_size([1.0, lam_ratio], [0.0, 0.0])
    assert n == 1024
    n, _ = oracle.image_size([1.0, lam_ratio * (1 + 1e-9)], [0.0, 0.0])
    assert n == 2048


def test_invalid():
    with pytest.raises(ValueError):
        oracle.image_size([0.0, 1.0], [0.0, 1.0])      # zero-length baseline
    with pytest.raises(ValueError):
        oracle.image_size([1.0], [1.0], f_max=2.0)      # criterion (i) needs f_max > 2


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_gpu_matches_oracle(dtype):
    import torch
    from paper_1709_06999_gb300 import Context, GalError
    ctx = Context(0)
    rng = np.random.default_rng(5)
    for m in (1, 7, 100_003):
        r = np.exp(rng.uniform(np.log(1e4), np.log(2e6), m))
        a = rng.uniform(0, 2 * np.pi, m)
        u = torch.tensor(r * np.cos(a), dtype=getattr(torch, dtype), device="cuda")
        v = torch.tensor(r * np.sin(a), dtype=getattr(torch, dtype), device="cuda")
        uh, vh = u.double().cpu().numpy(), v.double().cpu().numpy()   # the values the GPU sees
        for pb in (0.0, 1.5 * 1.3e-3 / 12.0, 1e-2):
            n_gpu, d_gpu = ctx.get_image_size(u, v, PB=pb)
            n_ref, d_ref = oracle.image_size(uh, vh, PB=pb)
            assert n_gpu == n_ref
            assert abs(d_gpu - d_ref) <= 1e-12 * d_ref
    # the table's ALMA C43-7 row through the device path
    lam = 1.3e-3
    u = torch.tensor([64.0 / lam, 0.0], dtype=torch.float64, device="cuda")
    v = torch.tensor([0.0, 3637.8 / lam], dtype=torch.float64, device="cuda")
    assert ctx.get_image_size(u, v)[0] == 1024
    assert ctx.get_image_size(u, v, PB=1.5 * lam / 12.0)[0] == 4096
    # a zero-length baseline or bad factors are rejected
    z = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(GalError):
        ctx.get_image_size(z, z)
    with pytest.raises(GalError):
        ctx.get_image_size(u, v, f_max=2.0)
