"""The host-side order of gal_data_create_sorted_* (gal_z_order_*), against a
plain restatement of its definition: both axes quantised to 16 bits over
[-rho, rho], the cells bit-interleaved (u in the even bits), a stable sort by
that key, points with a non-finite coordinate last.  No GPU needed."""
import numpy as np
import pytest

from paper_1709_06999_gb300 import _native


def _interleave(a, b):
    key = 0
    for bit in range(16):
        key |= ((a >> bit) & 1) << (2 * bit)
        key |= ((b >> bit) & 1) << (2 * bit + 1)
    return key


def _reference_order(u, v):
    u64, v64 = u.astype(np.float64), v.astype(np.float64)
    finite = np.isfinite(u64) & np.isfinite(v64)
    rho = float(np.sqrt(u64[finite] ** 2 + v64[finite] ** 2).max()) if finite.any() else 0.0
    scale = 65535.0 / (2.0 * rho) if rho > 0 else 0.0

    def cell(x):
        q = np.floor((x + rho) * scale)
        return int(min(max(q, 0.0), 65535.0))

    keys = [(_interleave(cell(a), cell(b)) if f else 0xFFFFFFFF)
            for a, b, f in zip(u64, v64, finite)]
    return sorted(range(len(keys)), key=lambda i: (keys[i], i)), keys


def _order(u, v, dt):
    lib = _native.load()
    fn = lib.gal_z_order_f32 if dt == np.float32 else lib.gal_z_order_f64
    u = np.ascontiguousarray(u, dtype=dt)
    v = np.ascontiguousarray(v, dtype=dt)
    perm = np.empty(u.size, dtype=np.int64)
    st = fn(u.ctypes.data, v.ctypes.data, u.size, perm.ctypes.data)
    assert st == 0
    return perm


@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_matches_definition(dt):
    rng = np.random.default_rng(11)
    n = 3001
    r = 10 ** rng.uniform(4, 6.5, n)
    a = rng.uniform(0, 2 * np.pi, n)
    u, v = (r * np.cos(a)).astype(dt), (r * np.sin(a)).astype(dt)
    u[5], v[9] = np.nan, np.inf           # non-finite points go last
    u[100:110] = u[50]                     # exact duplicates keep their input order
    v[100:110] = v[50]
    perm = _order(u, v, dt)
    ref, keys = _reference_order(u, v)
    assert perm.tolist() == ref
    assert sorted(perm.tolist()) == list(range(n))
    assert set(perm[-2:].tolist()) == {5, 9}
    k = np.array(keys, dtype=np.int64)[perm]
    assert np.all(np.diff(k) >= 0)


def test_neighbours_in_the_plane_are_neighbours_in_memory():
    # a regular 64 x 64 grid: consecutive stored points are mostly adjacent
    g = np.arange(64, dtype=np.float64) - 31.5
    u, v = np.meshgrid(g, g)
    perm = _order(u.ravel(), v.ravel(), np.float64)
    pu, pv = u.ravel()[perm], v.ravel()[perm]
    step = np.hypot(np.diff(pu), np.diff(pv))
    assert np.median(step) == 1.0
    assert np.mean(step) < 2.0


def test_edge_cases():
    lib = _native.load()
    perm = np.empty(1, dtype=np.int64)
    assert lib.gal_z_order_f64(None, None, 0, None) == 0
    assert lib.gal_z_order_f64(None, None, 1, perm.ctypes.data) != 0
    assert lib.gal_z_order_f64(None, None, -1, None) != 0
    zeros = np.zeros(4)
    assert _order(zeros, zeros, np.float64).tolist() == [0, 1, 2, 3]   # rho = 0: one cell
    nan = np.full(3, np.nan)
    assert _order(nan, nan, np.float64).tolist() == [0, 1, 2]
