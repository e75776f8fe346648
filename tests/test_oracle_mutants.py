"""Mutation test for the oracle's pins (CPU only).

Each mutant is a copy of the oracle source with one plausible mistake
planted in it (a dropped term, a flipped sign, a wrong or transposed index,
a missing shift).  The pins must reject every mutant: at least one check of
``pins.ALL_CHECKS`` has to fail on it.  The real oracle is never modified.
"""
import inspect
import types

import pytest

import pins
from oracle import galario_oracle as O

MUTANTS = {
    "no_input_shift": ("centred = np.fft.fftshift(img)", "centred = img"),
    "no_output_shift": ("return np.fft.fftshift(np.fft.rfft2(centred), axes=0)",
                        "return np.fft.rfft2(centred)"),
    "transposed_image": ("centred = np.fft.fftshift(img)", "centred = np.fft.fftshift(img.T)"),
    "phase_sign": ("return np.cos(theta) + 1j * np.sin(theta)",
                   "return np.cos(theta) - 1j * np.sin(theta)"),
    "no_conjugate_fold": ("vis = np.where(neg, np.conj(vis), vis)", "vis = vis"),
    "no_v_flip_fold": ("iv = nxy / 2.0 + np.where(neg, -vrot, vrot) / du", "iv = nxy / 2.0 + vrot / du"),
    "rotation_direction": ("return u * c - v * s, u * s + v * c", "return u * c + v * s, -u * s + v * c"),
    "offsets_not_rotated": ("dRA_rot = 2.0 * math.pi * (dRA * c - dDec * s)", "dRA_rot = 2.0 * math.pi * dRA"),
    "swapped_fractions": ("tv = fv - r0\n    tu = fu - c0", "tv = fu - c0\n    tu = fv - r0"),
    "wrong_corner": ("+ tv * (1.0 - tu) * G[r0 + 1, c0]\n", "+ tv * (1.0 - tu) * G[r0 + 1, c0 + 1]\n"),
    "v_index_off_by_one": ("iv = nxy / 2.0 + np.where", "iv = nxy / 2.0 - 1.0 + np.where"),
    "cell_size": ("    du = 1.0 / (nxy * dxy)\n    neg", "    du = 1.0 / ((nxy + 1) * dxy)\n    neg"),
    "signed_u_index": ("iu = np.abs(urot) / du", "iu = urot / du"),
    "chi2_no_weights": ("terms = np.asarray(w, dtype=np.float64) * (dr * dr + di * di)",
                        "terms = dr * dr + di * di"),
    "chi2_no_imag": ("terms = np.asarray(w, dtype=np.float64) * (dr * dr + di * di)",
                     "terms = np.asarray(w, dtype=np.float64) * (dr * dr)"),
    "sweep_no_pixel_area": ("img *= dxy * dxy", "pass"),
    "sweep_inclination_inverted": ("xs = x / math.cos(inc)", "xs = x * math.cos(inc)"),
    "sweep_transposed": ("r = np.sqrt(xs[None, :] ** 2 + y[:, None] ** 2)",
                         "r = np.sqrt(xs[:, None] ** 2 + y[None, :] ** 2)"),
    "sweep_no_centre": ("img[nxy // 2, nxy // 2] = centre * dxy * dxy", "pass"),
    "sweep_centre_not_extrapolated": ("centre = I[0] + slope * (0.0 - radii[0])", "centre = I[0]"),
    "pixel_origin_off_by_one": ("    half = nxy // 2\n    idx", "    half = nxy // 2 - 1\n    idx"),
    "size_gamma_half": ("MRS_GAMMA = 0.6", "MRS_GAMMA = 0.5"),
    "size_no_f_max": ("need = 2.0 * f_max * rho_max / duv", "need = 2.0 * rho_max / duv"),
    "size_iib_alone": ("duv = min(duv, 1.0 / PB)", "duv = 1.0 / PB"),
    "size_round_down": ("nxy = 2 ** (expo - 1) if mant == 0.5 else 2 ** expo", "nxy = 2 ** (expo - 1)"),
    "freq_wavelength_inverted": ("return (u_m * nu) / SPEED_OF_LIGHT, (v_m * nu) / SPEED_OF_LIGHT",
                                 "return (u_m / nu) * SPEED_OF_LIGHT, (v_m / nu) * SPEED_OF_LIGHT"),
    "multi_no_amplitude": ("        total = total + a * sample_image(image, dxy, u, v, x, y, PA)",
                           "        total = total + sample_image(image, dxy, u, v, x, y, PA)"),
    "multi_swapped_offsets": ("        total = total + a * sample_image(image, dxy, u, v, x, y, PA)",
                              "        total = total + a * sample_image(image, dxy, u, v, y, x, PA)"),
    "size_pixel_from_extent": ("return int(nxy), 1.0 / (nxy * duv)",
                               "return int(nxy), 1.0 / (2.0 * f_max * rho_max)"),
    "full_plane_u_not_shifted": ("return np.fft.fftshift(np.fft.fft2(np.fft.fftshift(img)))",
                                 "return np.fft.fftshift(np.fft.fft2(np.fft.fftshift(img)), axes=0)"),
    "full_plane_no_input_shift": ("return np.fft.fftshift(np.fft.fft2(np.fft.fftshift(img)))",
                                  "return np.fft.fftshift(np.fft.fft2(img))"),
    "full_plane_u_mirrored": ("iu = nxy / 2.0 + urot / du", "iu = nxy / 2.0 - urot / du"),
    "full_plane_conjugated": ("    vis = bilinear(Gf, iv, iu)\n", "    vis = np.conj(bilinear(Gf, iv, iu))\n"),
    "beam_centre_sign": ("sx = X * c + Y * s + dRA", "sx = X * c + Y * s - dRA"),
    "beam_rotation_direction": ("sx = X * c + Y * s + dRA\n    sy = -X * s + Y * c + dDec",
                                "sx = X * c - Y * s + dRA\n    sy = X * s + Y * c + dDec"),
    "beam_offsets_ignored": ("sy = -X * s + Y * c + dDec", "sy = -X * s + Y * c"),
    "beam_no_4ln2": ("np.exp(-FOUR_LN2 * (sx * sx + sy * sy) / (fwhm * fwhm))",
                     "np.exp(-(sx * sx + sy * sy) / (fwhm * fwhm))"),
    "beam_transposed": ("X = x[None, :]\n    Y = y[:, None]", "X = x[:, None]\n    Y = y[None, :]"),
}


def _mutant_module(name, old, new):
    src = inspect.getsource(O)
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    mod = types.ModuleType(f"oracle_mutant_{name}")
    exec(compile(src.replace(old, new), f"<mutant {name}>", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(name):
    mod = _mutant_module(name, *MUTANTS[name])
    failed = []
    for check in pins.ALL_CHECKS:
        try:
            check(mod)
        except (AssertionError, ValueError, IndexError, FloatingPointError):
            failed.append(check.__name__)
    assert failed, f"mutant {name} passes every pin"


def test_unmutated_source_passes():
    mod = _mutant_module("identity", "__all__ = [", "__all__ = [")
    for check in pins.ALL_CHECKS:
        check(mod)
