"""PyTorch-facing binding of the C ABI (argument marshalling only).

Tensors must live on the context's CUDA device; float32 tensors select the
``_f32`` entry points and float64 tensors the ``_f64`` ones.  Work is enqueued
on the current torch stream of that device.  Every computation happens in the
CUDA library; nothing here falls back to the CPU.

Names follow the paper's functions (Sect. 2): sweep, sample_image,
sample_profile, chi2_image, chi2_profile.
"""
from __future__ import annotations

import ctypes as ct

import torch

from . import _native

_SUFFIX = {torch.float32: "f32", torch.float64: "f64"}


class GalError(RuntimeError):
    pass


def _check(ctx_handle, status: int):
    if status != 0:
        lib = _native.load()
        msg = lib.gal_strerror(status).decode()
        if ctx_handle:
            cu = lib.gal_last_cuda_error(ctx_handle).decode()
            if cu:
                msg += f" ({cu})"
        raise GalError(f"galario_gb300 status {status}: {msg}")


def _opts(pb_fwhm: float, full_plane: bool):
    """gal_opts for the extended calls, or None when both are at their defaults."""
    if not pb_fwhm and not full_plane:
        return None
    return ct.byref(_native.GalOpts(float(pb_fwhm), 1 if full_plane else 0))


def _suffix(*tensors) -> str:
    dt = tensors[0].dtype
    if dt not in _SUFFIX:
        raise TypeError(f"unsupported dtype {dt}; use float32 or float64")
    for t in tensors[1:]:
        if t.dtype != dt:
            raise TypeError("all arrays of one call must share a dtype")
    return _SUFFIX[dt]


class Request:
    """One chi-square request of a batch: chi2Image (`image`) or chi2Profile
    (`intensity` and its sweep arguments), against a registered Observation."""

    def __init__(self, obs: "Observation", *, image=None, intensity=None, dxy: float,
                 nxy: int | None = None, dRA: float = 0.0, dDec: float = 0.0, PA: float = 0.0,
                 Rmin: float = 0.0, dR: float = 0.0, inc: float = 0.0, pb_fwhm: float = 0.0,
                 full_plane: bool = False):
        if (image is None) == (intensity is None):
            raise ValueError("give exactly one of image and intensity")
        self.obs, self.image, self.intensity = obs, image, intensity
        if image is not None:
            if image.dim() != 2 or image.shape[0] != image.shape[1]:
                raise ValueError("image must be square")
            nxy = image.shape[0]
        elif nxy is None:
            raise ValueError("a profile request needs nxy")
        self.nxy, self.dxy, self.dRA, self.dDec, self.PA = int(nxy), dxy, dRA, dDec, PA
        self.Rmin, self.dR, self.inc = Rmin, dR, inc
        self.pb_fwhm = pb_fwhm
        self.full_plane = bool(full_plane)

    def __setattr__(self, name, value):
        # any change of an argument drops the marshalled copy (_packed)
        object.__setattr__(self, "_packed", None)
        object.__setattr__(self, name, value)

    def _pack(self, ctx: "Context"):
        """The request as gal_request bytes and the tensor they point into.
        Reused while no argument was reassigned and the (contiguous) tensor
        still has the same storage on the context's device."""
        t = self.image if self.image is not None else self.intensity
        c = self._packed
        if (c is not None and c[0] == ctx.device and c[1] == t.data_ptr()
                and c[2] == self.obs.handle.value):  # an observation closed since: not reused
            return c[3], c[4]
        st, keep = self._struct(ctx)
        b = bytes(st)
        if keep is t:  # used in place, so its storage pointer identifies it
            object.__setattr__(self, "_packed",
                               (ctx.device, t.data_ptr(), self.obs.handle.value, b, keep))
        return b, keep

    def _struct(self, ctx: "Context"):
        dt = self.obs.dtype
        if self.image is not None:
            img = ctx._dev(self.image).contiguous()
            if img.dtype != dt:
                raise TypeError("image dtype must match the observation's")
            keep = img
            return _native.GalRequest(img.data_ptr(), None, 0, 0.0, 0.0, 0.0, self.nxy, self.dxy,
                                      self.dRA, self.dDec, self.PA, self.obs.handle.value,
                                      self.pb_fwhm, int(self.full_plane)), keep
        I = ctx._dev(self.intensity).contiguous()
        if I.dtype != dt:
            raise TypeError("intensity dtype must match the observation's")
        return _native.GalRequest(None, I.data_ptr(), I.numel(), self.Rmin, self.dR, self.inc,
                                  self.nxy, self.dxy, self.dRA, self.dDec, self.PA,
                                  self.obs.handle.value, self.pb_fwhm, int(self.full_plane)), I


def _request_array(ctx, requests):
    parts, keep = [], []
    for r in requests:
        b, k = r._pack(ctx)
        parts.append(b)
        keep.append(k)
    size = ct.sizeof(_native.GalRequest)
    data = b"".join(parts) if parts else bytes(size)
    arr = (_native.GalRequest * max(1, len(parts))).from_buffer_copy(data)
    return arr, keep


class BatchGraph:
    """A batch recorded into a CUDA graph (gal_chi2_batch_capture).  `out`
    receives the chi-squares at every launch; the graph reads the requests'
    tensors as they are when it runs."""

    def __init__(self, ctx: "Context", requests, out):
        self.ctx, self.out = ctx, out
        arr, self._keep = _request_array(ctx, requests)
        h = ct.c_void_p()
        _check(ctx.handle, ctx.lib.gal_chi2_batch_capture(ctx.handle, arr, len(requests),
                                                          out.data_ptr(), ctx._stream(),
                                                          ct.byref(h)))
        self.handle = h.value

    def launch(self):
        _check(self.ctx.handle, self.ctx.lib.gal_graph_launch(self.handle, self.ctx._stream()))
        return self.out

    def update(self, requests):
        arr, keep = _request_array(self.ctx, requests)
        _check(self.ctx.handle, self.ctx.lib.gal_graph_update(self.handle, arr, len(requests),
                                                              self.out.data_ptr()))
        self._keep = keep

    def close(self):
        if getattr(self, "handle", None):
            self.ctx.lib.gal_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Observation:
    """A registered set of M visibilities (u, v, Re, Im, w) resident on the device.

    Holds references to its tensors so that the borrowed device memory stays
    alive.  Creation enqueues one reduction for the uv extent.
    """

    def __init__(self, ctx: "Context", u, v, re, im, w, nu=None, z_order=False):
        """u, v in wavelengths; or, with `nu` (Hz per visibility), in metres
        (gal_data_create_freq_*: the library converts them once).  z_order:
        the library keeps copies in Z-order of the uv plane
        (gal_data_create_sorted_*), the tensors are not kept."""
        if z_order and nu is not None:
            raise ValueError("z_order applies to observations in wavelengths")
        arrays = (u, v, re, im, w) if nu is None else (u, v, nu, re, im, w)
        tensors = [ctx._dev(t).contiguous() for t in arrays]
        m = tensors[0].numel()
        if any(t.numel() != m for t in tensors):
            raise ValueError("u, v, re, im, w (and nu) must have the same length")
        self.ctx = ctx
        self.M = m
        self.dtype = tensors[0].dtype
        sfx = _suffix(*tensors)
        h = ct.c_void_p()
        name = (f"gal_data_create_freq_{sfx}" if nu is not None else
                f"gal_data_create_sorted_{sfx}" if z_order else f"gal_data_create_{sfx}")
        fn = getattr(ctx.lib, name)
        _check(ctx.handle, fn(ctx.handle, *[t.data_ptr() for t in tensors], m, ctx._stream(), ct.byref(h)))
        self.handle = h
        # borrowed arrays stay alive with the handle (with nu, u and v live in
        # the library)
        self._tensors = [] if z_order else tensors if nu is None else tensors[3:]

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            self.ctx.lib.gal_data_destroy(self.handle)
            self.handle = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """Owns the library workspace on one CUDA device."""

    def __init__(self, device: int = 0):
        self.lib = _native.load()
        self.device = torch.device("cuda", device)
        h = ct.c_void_p()
        _check(None, self.lib.gal_create(ct.byref(h), device))
        self.handle = h

    # -- plumbing -----------------------------------------------------------
    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            self.lib.gal_destroy(self.handle)
            self.handle = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream(self) -> int:
        # the library enqueues on the calling thread's current device
        if torch.cuda.current_device() != self.device.index:
            raise GalError(f"current CUDA device is {torch.cuda.current_device()}, the context's "
                           f"is {self.device.index}: select it first (torch.cuda.set_device)")
        return torch.cuda.current_stream(self.device).cuda_stream

    def _dev(self, t):
        if not isinstance(t, torch.Tensor):
            raise TypeError("expected a torch.Tensor")
        if t.device != self.device:
            raise ValueError(f"tensor on {t.device}, context on {self.device}")
        return t.contiguous()

    def workspace_bytes(self) -> int:
        """Device workspace this context holds now (gal_workspace_bytes)."""
        return int(self.lib.gal_workspace_bytes(self.handle))

    def set_hbm_budget(self, nbytes: int):
        """Limit this context's workspace to nbytes (0: no limit); a call that
        would exceed it raises GalError (GAL_E_NOMEM) without evaluating."""
        _check(self.handle, self.lib.gal_set_hbm_budget(self.handle, int(nbytes)))

    def reserve(self, nxy: int, dtype=torch.float32):
        _check(self.handle, self.lib.gal_reserve(self.handle, nxy, 4 if dtype == torch.float32 else 8))

    def check(self):
        _check(self.handle, self.lib.gal_check(self.handle))

    def launch_count(self) -> int:
        return int(self.lib.gal_launch_count(self.handle))

    def set_stage_timing(self, enable=True, stages=None):
        """Time every stage (enable=True), none (False), or only the stage
        indices in `stages` (0 extent, 1 row FFT, 2 column FFT, 3 sample/chi2)."""
        mask = 0xF if enable else 0
        if enable and stages is not None:
            mask = sum(1 << int(s) for s in set(stages))
        _check(self.handle, self.lib.gal_set_stage_timing(self.handle, mask))

    def stage_times(self):
        """Per stage (extent, row FFT, column FFT, sample/chi2): (total ms, launches)."""
        ms = (ct.c_double * 4)()
        n = (ct.c_int64 * 4)()
        _check(self.handle, self.lib.gal_stage_times(self.handle, ms, n))
        return [(ms[i], n[i]) for i in range(4)]

    def register_freq(self, u_m, v_m, nu, re, im, w) -> Observation:
        """Register visibilities with baselines in metres and their frequencies (Hz)."""
        return Observation(self, u_m, v_m, re, im, w, nu=nu)

    def register(self, u, v, re, im, w, z_order: bool = False) -> Observation:
        """Register visibilities (u, v in wavelengths).  z_order=True keeps
        library-owned copies ordered along the uv plane (faster gathers from
        spectra too large for shared memory; chi-square equal up to rounding)."""
        return Observation(self, u, v, re, im, w, z_order=z_order)

    # -- operations ---------------------------------------------------------
    def sweep(self, intensity, Rmin: float, dR: float, nxy: int, dxy: float, inc: float = 0.0,
              out=None):
        I = self._dev(intensity)
        sfx = _suffix(I)
        if out is None:
            out = torch.empty((nxy, nxy), dtype=I.dtype, device=self.device)
        fn = getattr(self.lib, f"gal_sweep_{sfx}")
        _check(self.handle, fn(self.handle, I.data_ptr(), I.numel(), Rmin, dR, nxy, dxy, inc,
                               out.data_ptr(), self._stream()))
        return out

    def sample_image(self, image, dxy: float, u, v, dRA: float = 0.0, dDec: float = 0.0,
                     PA: float = 0.0, out=None, *, pb_fwhm: float = 0.0, full_plane: bool = False):
        """Visibilities as an (M, 2) tensor of (Re, Im).  pb_fwhm > 0 applies a
        primary beam of that FWHM (radians); full_plane uses the
        complex-to-complex spectrum (gal_opts)."""
        img, u, v = self._dev(image), self._dev(u), self._dev(v)
        sfx = _suffix(img, u, v)
        nxy = img.shape[0]
        if img.dim() != 2 or img.shape[1] != nxy:
            raise ValueError("image must be square")
        m = u.numel()
        if out is None:
            out = torch.empty((m, 2), dtype=img.dtype, device=self.device)
        opts = _opts(pb_fwhm, full_plane)
        head = (self.handle, img.data_ptr(), nxy, dxy, dRA, dDec, PA)
        tail = (m, u.data_ptr(), v.data_ptr(), out.data_ptr(), self._stream())
        if opts is None:
            _check(self.handle, getattr(self.lib, f"gal_sample_image_{sfx}")(*head, *tail))
        else:
            _check(self.handle, getattr(self.lib, f"gal_sample_image_ex_{sfx}")(*head, opts, *tail))
        return out

    def sample_profile(self, intensity, Rmin: float, dR: float, nxy: int, dxy: float, u, v,
                       inc: float = 0.0, dRA: float = 0.0, dDec: float = 0.0, PA: float = 0.0,
                       out=None, *, pb_fwhm: float = 0.0, full_plane: bool = False):
        I, u, v = self._dev(intensity), self._dev(u), self._dev(v)
        sfx = _suffix(I, u, v)
        m = u.numel()
        if out is None:
            out = torch.empty((m, 2), dtype=I.dtype, device=self.device)
        opts = _opts(pb_fwhm, full_plane)
        head = (self.handle, I.data_ptr(), I.numel(), Rmin, dR, nxy, dxy, inc, dRA, dDec, PA)
        tail = (m, u.data_ptr(), v.data_ptr(), out.data_ptr(), self._stream())
        if opts is None:
            _check(self.handle, getattr(self.lib, f"gal_sample_profile_{sfx}")(*head, *tail))
        else:
            _check(self.handle,
                   getattr(self.lib, f"gal_sample_profile_ex_{sfx}")(*head, opts, *tail))
        return out

    def chi2_image(self, image, dxy: float, obs: Observation, dRA: float = 0.0, dDec: float = 0.0,
                   PA: float = 0.0, out=None, *, pb_fwhm: float = 0.0, full_plane: bool = False):
        """chi2 as a one-element float64 device tensor (stream-ordered, no sync)."""
        img = self._dev(image)
        sfx = _suffix(img)
        if out is None:
            out = torch.empty((), dtype=torch.float64, device=self.device)
        opts = _opts(pb_fwhm, full_plane)
        head = (self.handle, img.data_ptr(), img.shape[0], dxy, dRA, dDec, PA)
        tail = (obs.handle, out.data_ptr(), self._stream())
        if opts is None:
            _check(self.handle, getattr(self.lib, f"gal_chi2_image_{sfx}")(*head, *tail))
        else:
            _check(self.handle, getattr(self.lib, f"gal_chi2_image_ex_{sfx}")(*head, opts, *tail))
        return out

    def chi2_profile(self, intensity, Rmin: float, dR: float, nxy: int, dxy: float,
                     obs: Observation, inc: float = 0.0, dRA: float = 0.0, dDec: float = 0.0,
                     PA: float = 0.0, out=None, *, pb_fwhm: float = 0.0,
                     full_plane: bool = False):
        I = self._dev(intensity)
        sfx = _suffix(I)
        if out is None:
            out = torch.empty((), dtype=torch.float64, device=self.device)
        opts = _opts(pb_fwhm, full_plane)
        head = (self.handle, I.data_ptr(), I.numel(), Rmin, dR, nxy, dxy, inc, dRA, dDec, PA)
        tail = (obs.handle, out.data_ptr(), self._stream())
        if opts is None:
            _check(self.handle, getattr(self.lib, f"gal_chi2_profile_{sfx}")(*head, *tail))
        else:
            _check(self.handle,
                   getattr(self.lib, f"gal_chi2_profile_ex_{sfx}")(*head, opts, *tail))
        return out

    def chi2_image_host_async(self, image_host, dxy: float, obs: Observation, out, index: int = 0,
                              dRA: float = 0.0, dDec: float = 0.0, PA: float = 0.0):
        """Enqueue chi2Image of a host image (pinned) without waiting: its copy
        overlaps the previous call's compute; the result lands in out[index]
        (a pinned float64 CPU tensor) once the current stream reaches this call.
        Neither the image nor out may be touched before then."""
        if image_host.device.type != "cpu" or out.device.type != "cpu":
            raise ValueError("image_host and out must be CPU tensors")
        if out.dtype != torch.float64 or not out.is_contiguous() or not 0 <= index < out.numel():
            raise ValueError("out must be a contiguous float64 tensor with room for index")
        if not image_host.is_contiguous():
            raise ValueError("image_host must be contiguous (it is read after this call returns)")
        sfx = _suffix(image_host)
        fn = getattr(self.lib, f"gal_chi2_image_host_async_{sfx}")
        _check(self.handle, fn(self.handle, image_host.data_ptr(), image_host.shape[0], dxy, dRA,
                               dDec, PA, obs.handle, out.data_ptr() + 8 * index, self._stream()))
        return out

    def chi2_image_host(self, image_host, dxy: float, obs: Observation, dRA: float = 0.0,
                        dDec: float = 0.0, PA: float = 0.0) -> float:
        """chi2Image from a host (ideally pinned) image; copies in, computes, copies back."""
        if image_host.device.type != "cpu":
            raise ValueError("image_host must be a CPU tensor")
        img = image_host.contiguous()
        sfx = _suffix(img)
        res = ct.c_double()
        fn = getattr(self.lib, f"gal_chi2_image_host_{sfx}")
        _check(self.handle, fn(self.handle, img.data_ptr(), img.shape[0], dxy, dRA, dDec, PA,
                               obs.handle, ct.byref(res), self._stream()))
        return res.value

    # -- multi-source composition (K offset copies of one model) -------------
    @staticmethod
    def _sources(dRA, dDec, amp):
        dRA = [float(x) for x in dRA]
        dDec = [float(x) for x in dDec]
        amp = [1.0] * len(dRA) if amp is None else [float(x) for x in amp]
        if not (len(dRA) == len(dDec) == len(amp)):
            raise ValueError("dRA, dDec and amp must have the same length")
        arr = lambda xs: (ct.c_double * max(1, len(xs)))(*xs)  # noqa: E731
        return len(dRA), arr(dRA), arr(dDec), arr(amp)

    def sample_image_multi(self, image, dxy: float, u, v, dRA, dDec, amp=None, PA: float = 0.0,
                           out=None):
        """Visibilities of K copies of `image`, copy k scaled by amp[k] and
        shifted by (dRA[k], dDec[k]), all rotated by PA: one FFT for all."""
        img, u, v = self._dev(image), self._dev(u), self._dev(v)
        sfx = _suffix(img, u, v)
        K, a, b, c = self._sources(dRA, dDec, amp)
        m = u.numel()
        if out is None:
            out = torch.empty((m, 2), dtype=img.dtype, device=self.device)
        fn = getattr(self.lib, f"gal_sample_image_multi_{sfx}")
        _check(self.handle, fn(self.handle, img.data_ptr(), img.shape[0], dxy, PA, K, a, b, c, m,
                               u.data_ptr(), v.data_ptr(), out.data_ptr(), self._stream()))
        return out

    def chi2_image_multi(self, image, dxy: float, obs: Observation, dRA, dDec, amp=None,
                         PA: float = 0.0, out=None):
        img = self._dev(image)
        sfx = _suffix(img)
        K, a, b, c = self._sources(dRA, dDec, amp)
        if out is None:
            out = torch.empty((), dtype=torch.float64, device=self.device)
        fn = getattr(self.lib, f"gal_chi2_image_multi_{sfx}")
        _check(self.handle, fn(self.handle, img.data_ptr(), img.shape[0], dxy, PA, K, a, b, c,
                               obs.handle, out.data_ptr(), self._stream()))
        return out

    def chi2_profile_multi(self, intensity, Rmin: float, dR: float, nxy: int, dxy: float,
                           obs: Observation, dRA, dDec, amp=None, inc: float = 0.0,
                           PA: float = 0.0, out=None):
        I = self._dev(intensity)
        sfx = _suffix(I)
        K, a, b, c = self._sources(dRA, dDec, amp)
        if out is None:
            out = torch.empty((), dtype=torch.float64, device=self.device)
        fn = getattr(self.lib, f"gal_chi2_profile_multi_{sfx}")
        _check(self.handle, fn(self.handle, I.data_ptr(), I.numel(), Rmin, dR, nxy, dxy, inc, PA,
                               K, a, b, c, obs.handle, out.data_ptr(), self._stream()))
        return out

    def chi2_batch(self, requests, out=None):
        """chi-square of every Request, as a float64 tensor of len(requests)
        (gal_chi2_batch: shared launches per pass and image side)."""
        n = len(requests)
        if out is None:
            out = torch.empty(n, dtype=torch.float64, device=self.device)
        arr, keep = _request_array(self, requests)
        _check(self.handle, self.lib.gal_chi2_batch(self.handle, arr, n, out.data_ptr(),
                                                    self._stream()))
        del keep
        return out

    def set_batch_tuning(self, enable: bool):
        _check(self.handle, self.lib.gal_set_batch_tuning(self.handle, int(enable)))

    def set_batch_shape(self, dtype, n: int, max_nxy: int, row_blocks: int,
                        jobs_per_launch: int, gather_fold: int):
        """Fix the launch shape of batches with n requests of this precision
        in the batched kernels, largest side max_nxy (gal_set_batch_shape)."""
        _check(self.handle, self.lib.gal_set_batch_shape(
            self.handle, _real_bytes(dtype), int(n), int(max_nxy), int(row_blocks),
            int(jobs_per_launch), int(gather_fold)))

    def batch_shape(self, dtype, n: int, max_nxy: int):
        """((row_blocks, jobs_per_launch, gather_fold), kept) for that batch
        key: the shape its next batch uses, and whether it was tuned or set
        (gal_get_batch_shape)."""
        sh = (ct.c_int * 3)()
        kept = ct.c_int()
        _check(self.handle, self.lib.gal_get_batch_shape(self.handle, _real_bytes(dtype), int(n),
                                                         int(max_nxy), sh, ct.byref(kept)))
        return (sh[0], sh[1], sh[2]), bool(kept.value)

    def capture_batch(self, requests, out=None) -> BatchGraph:
        if out is None:
            out = torch.empty(len(requests), dtype=torch.float64, device=self.device)
        return BatchGraph(self, requests, out)

    def get_image_size(self, u, v, PB: float = 0.0, f_min: float = 5.0, f_max: float = 2.5):
        """(nxy, dxy) for the uv points (Sect. 3.3): criterion (iia) when PB == 0,
        (iib) with PB the primary-beam FWHM in radians otherwise."""
        u, v = self._dev(u), self._dev(v)
        sfx = _suffix(u, v)
        if u.numel() != v.numel():
            raise ValueError("u and v must have the same length")
        n = ct.c_int64()
        d = ct.c_double()
        fn = getattr(self.lib, f"gal_get_image_size_{sfx}")
        _check(self.handle, fn(self.handle, u.data_ptr(), v.data_ptr(), u.numel(), PB, f_min,
                               f_max, ct.byref(n), ct.byref(d), self._stream()))
        return n.value, d.value


class ServedData:
    """An observation held by a Server (borrowed tensors kept alive here;
    none when the server keeps its own copies)."""

    def __init__(self, handle, tensors, dtype):
        self.handle = handle
        self._tensors = tensors
        self.dtype = dtype


class Server:
    """The request loop of gal_server_*: a FIFO of chi-square requests served
    by `slots` worker contexts under an HBM budget, with queued requests of
    one precision admitted together as one batch (up to max_batch)."""

    def __init__(self, device: int = 0, hbm_budget: int = 150 * 10**9, slots: int = 4,
                 max_batch: int = 16):
        self.lib = _native.load()
        self.device = torch.device("cuda", device)
        h = ct.c_void_p()
        _check(None, self.lib.gal_server_create(device, int(hbm_budget), slots, max_batch,
                                                ct.byref(h)))
        self.handle = h.value
        self._data = []
        self._inflight = {}

    def add_data(self, u, v, re, im, w, z_order: bool = False) -> ServedData:
        """Register an observation for requests (charged to the budget);
        z_order=True keeps library copies ordered along the uv plane."""
        tensors = [t.to(self.device).contiguous() for t in (u, v, re, im, w)]
        m = tensors[0].numel()
        if any(t.numel() != m for t in tensors):
            raise ValueError("u, v, re, im, w must have the same length")
        sfx = _suffix(*tensors)
        h = ct.c_void_p()
        name = f"gal_server_add_data_sorted_{sfx}" if z_order else f"gal_server_add_data_{sfx}"
        fn = getattr(self.lib, name)
        _check(None, fn(self.handle, *[t.data_ptr() for t in tensors], m, ct.byref(h)))
        d = ServedData(ct.c_void_p(h.value), [] if z_order else tensors, tensors[0].dtype)
        self._data.append(d)
        return d

    def _struct(self, req: "Request"):
        if req.image is not None:
            t = req.image.to(self.device).contiguous()
            st = _native.GalRequest(t.data_ptr(), None, 0, 0.0, 0.0, 0.0, req.nxy, req.dxy,
                                    req.dRA, req.dDec, req.PA, req.obs.handle.value, req.pb_fwhm, int(req.full_plane))
        else:
            t = req.intensity.to(self.device).contiguous()
            st = _native.GalRequest(None, t.data_ptr(), t.numel(), req.Rmin, req.dR, req.inc,
                                    req.nxy, req.dxy, req.dRA, req.dDec, req.PA,
                                    req.obs.handle.value, req.pb_fwhm, int(req.full_plane))
        if t.dtype != req.obs.dtype:
            raise TypeError("model dtype must match the observation's")
        return st, t

    def submit(self, req: "Request") -> int:
        """Queue a Request whose `obs` is a ServedData; returns its ticket."""
        st, t = self._struct(req)
        tk = ct.c_uint64()
        _check(None, self.lib.gal_server_submit(self.handle, ct.byref(st), ct.byref(tk)))
        self._inflight[tk.value] = t           # keep the model alive until collected
        return tk.value

    def submit_many(self, reqs) -> list:
        """Queue several Requests at once (they reach the queue together)."""
        pairs = [self._struct(r) for r in reqs]
        arr = (_native.GalRequest * max(1, len(pairs)))(*[p[0] for p in pairs])
        tks = (ct.c_uint64 * max(1, len(pairs)))()
        _check(None, self.lib.gal_server_submit_many(self.handle, arr, len(pairs), tks))
        for k, (_, t) in enumerate(pairs):
            self._inflight[tks[k]] = t
        return [tks[k] for k in range(len(pairs))]

    def wait(self, ticket: int, timeout_ms: int = -1):
        """(chi2, latency in seconds) of a ticket."""
        c, lat = ct.c_double(), ct.c_double()
        st = self.lib.gal_server_wait(self.handle, ticket, timeout_ms, ct.byref(c), ct.byref(lat))
        if st != -7:
            self._inflight.pop(ticket, None)
        _check(None, st)
        return c.value, lat.value

    def stats(self) -> dict:
        s = _native.GalServerStats()
        _check(None, self.lib.gal_server_get_stats(self.handle, ct.byref(s)))
        return {k: getattr(s, k) for k, _ in s._fields_}

    def close(self):
        if getattr(self, "handle", None):
            self.lib.gal_server_destroy(self.handle)
            self.handle = None
            self._inflight.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _real_bytes(dtype) -> int:
    if dtype in (torch.float32, "float32", "f32", 4):
        return 4
    if dtype in (torch.float64, "float64", "f64", 8):
        return 8
    raise ValueError(f"dtype must be float32 or float64, got {dtype!r}")


def set_fft_radix(device: int, dtype, nxy: int, row_radix: int, col_radix: int) -> None:
    """Fix the FFT plan of image side nxy (radix of the row and the column
    pass: 16 or 8 for float32 sides 32..512; 16 above; 8 for float64) on a
    device for this process; see gal_set_fft_radix."""
    lib = _native.load()
    _check(None, lib.gal_set_fft_radix(int(device), _real_bytes(dtype), int(nxy), int(row_radix),
                                       int(col_radix)))


def get_fft_radix(device: int, dtype, nxy: int):
    """(row radix, column radix) of side nxy on a device, or (0, 0) while no
    call has fixed it."""
    lib = _native.load()
    r, c = ct.c_int(), ct.c_int()
    _check(None, lib.gal_get_fft_radix(int(device), _real_bytes(dtype), int(nxy), ct.byref(r),
                                       ct.byref(c)))
    return r.value, c.value


_default: dict[int, Context] = {}


def default_context(device: int | None = None) -> Context:
    d = torch.cuda.current_device() if device is None else device
    if d not in _default:
        _default[d] = Context(d)
    return _default[d]


# -- the paper's calling convention (Sect. 2), on the default context --------
def sample_image(image, dxy, u, v, dRA=0.0, dDec=0.0, PA=0.0):
    return default_context(image.device.index).sample_image(image, dxy, u, v, dRA, dDec, PA)


def sample_profile(intensity, Rmin, dR, nxy, dxy, u, v, dRA=0.0, dDec=0.0, PA=0.0, inc=0.0):
    return default_context(intensity.device.index).sample_profile(
        intensity, Rmin, dR, nxy, dxy, u, v, inc, dRA, dDec, PA)


def chi2_image(image, dxy, u, v, re, im, w, dRA=0.0, dDec=0.0, PA=0.0):
    ctx = default_context(image.device.index)
    obs = ctx.register(u, v, re, im, w)
    return ctx.chi2_image(image, dxy, obs, dRA, dDec, PA)


def chi2_profile(intensity, Rmin, dR, nxy, dxy, u, v, re, im, w, dRA=0.0, dDec=0.0, PA=0.0,
                 inc=0.0):
    ctx = default_context(intensity.device.index)
    obs = ctx.register(u, v, re, im, w)
    return ctx.chi2_profile(intensity, Rmin, dR, nxy, dxy, obs, inc, dRA, dDec, PA)


def sweep(intensity, Rmin, dR, nxy, dxy, inc=0.0):
    return default_context(intensity.device.index).sweep(intensity, Rmin, dR, nxy, dxy, inc)


def get_image_size(u, v, PB=0.0, f_min=5.0, f_max=2.5):
    return default_context(u.device.index).get_image_size(u, v, PB, f_min, f_max)
