"""Host-side marshalling of batch requests (no GPU): the packed gal_request
bytes a Request keeps between calls follow every change of its arguments."""
import ctypes as ct

import torch

from paper_1709_06999_gb300 import _native, api


class _Obs:
    dtype = torch.float32

    def __init__(self, h):
        self.handle = ct.c_void_p(h)


class _Ctx:
    device = torch.device("cpu")

    def _dev(self, t):
        return t.contiguous()


def _arr(reqs):
    arr, keep = api._request_array(_Ctx(), reqs)
    return arr, keep


def test_fields_and_reuse():
    imgs = [torch.zeros(16, 16) for _ in range(3)]
    obs = _Obs(1234)
    reqs = [api.Request(obs, image=im, dxy=1e-8, dRA=1e-7 * k, PA=0.1) for k, im in enumerate(imgs)]
    arr, keep = _arr(reqs)
    assert [arr[k].image for k in range(3)] == [im.data_ptr() for im in imgs]
    assert arr[2].dRA == 2e-7 and arr[1].nxy == 16 and arr[0].data == 1234
    assert all(k is im for k, im in zip(keep, imgs))
    assert reqs[1]._packed is not None          # kept for the next call
    again, _ = _arr(reqs)
    assert bytes(again) == bytes(arr)


def test_reassigned_argument_is_repacked():
    im = torch.zeros(8, 8)
    r = api.Request(_Obs(7), image=im, dxy=1e-8, dRA=1e-7)
    _arr([r])
    r.dRA = 3e-7
    r.pb_fwhm = 1e-4
    arr, _ = _arr([r])
    assert arr[0].dRA == 3e-7 and arr[0].pb_fwhm == 1e-4
    other = torch.ones(8, 8)
    r.image = other
    arr, _ = _arr([r])
    assert arr[0].image == other.data_ptr()


def test_new_storage_and_closed_observation_are_repacked():
    im = torch.zeros(8, 8)
    obs = _Obs(99)
    r = api.Request(obs, image=im, dxy=1e-8)
    _arr([r])
    im.set_(torch.zeros(8, 8).untyped_storage(), 0, (8, 8))  # same tensor, new storage
    arr, _ = _arr([r])
    assert arr[0].image == im.data_ptr()
    obs.handle = ct.c_void_p()  # what Observation.close() leaves
    arr, _ = _arr([r])
    assert not arr[0].data


def test_non_contiguous_tensor_is_not_kept():
    base = torch.zeros(8, 16)
    im = base[:, ::2]
    r = api.Request(_Obs(5), image=im, dxy=1e-8)
    arr, keep = _arr([r])
    assert r._packed is None and keep[0] is not im and arr[0].image == keep[0].data_ptr()


def test_empty_list_gives_one_zeroed_struct():
    arr, keep = _arr([])
    assert len(arr) == 1 and keep == [] and not arr[0].image and arr[0].nxy == 0
    assert ct.sizeof(arr) == ct.sizeof(_native.GalRequest)
