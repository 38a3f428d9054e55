"""Python binding of the C ABI: torch tensors in, torch tensors out.

PyTorch provides device memory and the current CUDA stream; every step of protect and
restore runs in the library's CUDA kernels.  Function names follow include/fds.h.
"""
from __future__ import annotations

import ctypes
import functools
import json
import math
import os
from dataclasses import dataclass
from typing import Sequence

import torch

from . import _lib


def _stream_ptr(device: torch.device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _check_key(b: bytes, what: str) -> bytes:
    b = bytes(b)
    if len(b) != 16:
        raise ValueError(f"{what} must be 16 bytes")
    return b


def init(device: int = 0) -> None:
    """fds_init: select the device and build the library's device tables."""
    _lib.check(_lib.load().fds_init(device), "fds_init")


@functools.lru_cache(maxsize=8192)
def sizes(width: int, height: int, k: int) -> tuple[int, int]:
    """fds_sizes: (public bytes, private bytes) of one image (remembered per shape)."""
    pub, priv = ctypes.c_uint64(), ctypes.c_uint64()
    _lib.check(_lib.load().fds_sizes(width, height, k, ctypes.byref(pub), ctypes.byref(priv)),
               "fds_sizes")
    return pub.value, priv.value


def key_register(key: bytes) -> int:
    """fds_key_register: keep an AES-128 key's round keys resident; returns its slot."""
    slot = ctypes.c_int32()
    _lib.check(_lib.load().fds_key_register(_check_key(key, "key"), ctypes.byref(slot)),
               "fds_key_register")
    return slot.value


def key_release(slot: int) -> None:
    _lib.check(_lib.load().fds_key_release(slot), "fds_key_release")


def _image_dims(pixels: torch.Tensor) -> tuple[int, int]:
    if pixels.dtype != torch.uint8 or pixels.dim() != 3 or pixels.shape[2] != 3:
        raise ValueError("pixels must be an H x W x 3 uint8 tensor")
    if not pixels.is_cuda or not pixels.is_contiguous():
        raise ValueError("pixels must be a contiguous CUDA tensor")
    return int(pixels.shape[1]), int(pixels.shape[0])


def protect_image(pixels: torch.Tensor, key: bytes, iv: bytes, k: int,
                  public_out: torch.Tensor | None = None,
                  private_out: torch.Tensor | None = None) -> tuple[torch.Tensor, torch.Tensor]:
    """fds_protect_image: returns (public int16 [H/8, W/8, 3, 63-k], private uint8 bytes)."""
    w, h = _image_dims(pixels)
    pub_b, priv_b = sizes(w, h, k)
    dev = pixels.device
    if public_out is None:
        public_out = torch.empty((h // 8, w // 8, 3, 63 - k), dtype=torch.int16, device=dev)
    if private_out is None:
        private_out = torch.empty(priv_b, dtype=torch.uint8, device=dev)
    assert public_out.numel() * 2 == pub_b and private_out.numel() == priv_b
    rc = _lib.load().fds_protect_image(
        pixels.data_ptr(), w, h, k, _check_key(key, "key"), _check_key(iv, "iv"),
        public_out.data_ptr() if public_out.numel() else None, private_out.data_ptr(),
        _stream_ptr(dev))
    _lib.check(rc, "fds_protect_image")
    return public_out, private_out


TC_FORMS = {"bf16": _lib.FDS_TC_BF16, "tf32": _lib.FDS_TC_TF32, "f16": _lib.FDS_TC_F16}


def _tc_form(form: str) -> int:
    if form not in TC_FORMS:
        raise ValueError(f"form must be one of {sorted(TC_FORMS)}")
    return TC_FORMS[form]


def protect_image_tc(pixels: torch.Tensor, key: bytes, iv: bytes, k: int, form: str = "bf16",
                     public_out: torch.Tensor | None = None,
                     private_out: torch.Tensor | None = None) -> tuple[torch.Tensor, torch.Tensor]:
    """fds_protect_image_tc: the tensor-core precision form ("bf16" three-limb or "tf32"
    two-limb basis split); same outputs as protect_image, bit for bit."""
    f = _tc_form(form)
    w, h = _image_dims(pixels)
    pub_b, priv_b = sizes(w, h, k)
    dev = pixels.device
    if public_out is None:
        public_out = torch.empty((h // 8, w // 8, 3, 63 - k), dtype=torch.int16, device=dev)
    if private_out is None:
        private_out = torch.empty(priv_b, dtype=torch.uint8, device=dev)
    assert public_out.numel() * 2 == pub_b and private_out.numel() == priv_b
    rc = _lib.load().fds_protect_image_tc(
        f, pixels.data_ptr(), w, h, k, _check_key(key, "key"), _check_key(iv, "iv"),
        public_out.data_ptr() if public_out.numel() else None, private_out.data_ptr(),
        _stream_ptr(dev))
    _lib.check(rc, "fds_protect_image_tc")
    return public_out, private_out


def restore_image(public: torch.Tensor, private: torch.Tensor, width: int, height: int, k: int,
                  key: bytes, iv: bytes, pixels_out: torch.Tensor | None = None) -> torch.Tensor:
    """fds_restore_image: returns the H x W x 3 uint8 image."""
    dev = private.device
    if pixels_out is None:
        pixels_out = torch.empty((height, width, 3), dtype=torch.uint8, device=dev)
    rc = _lib.load().fds_restore_image(
        public.data_ptr() if public.numel() else None, private.data_ptr(), width, height, k,
        _check_key(key, "key"), _check_key(iv, "iv"), pixels_out.data_ptr(), _stream_ptr(dev))
    _lib.check(rc, "fds_restore_image")
    return pixels_out


def restore_image_tc(public: torch.Tensor, private: torch.Tensor, width: int, height: int, k: int,
                     key: bytes, iv: bytes, pixels_out: torch.Tensor | None = None,
                     form: str = "f16") -> torch.Tensor:
    """fds_restore_image_tc: restore with the inverse transform on tensor cores (form "f16");
    the same H x W x 3 uint8 image as restore_image, bit for bit."""
    f = _tc_form(form)
    dev = private.device
    if pixels_out is None:
        pixels_out = torch.empty((height, width, 3), dtype=torch.uint8, device=dev)
    rc = _lib.load().fds_restore_image_tc(
        f, public.data_ptr() if public.numel() else None, private.data_ptr(), width, height, k,
        _check_key(key, "key"), _check_key(iv, "iv"), pixels_out.data_ptr(), _stream_ptr(dev))
    _lib.check(rc, "fds_restore_image_tc")
    return pixels_out


@dataclass
class ImageDesc:
    """One image of a batch (struct fds_image): byte offsets into the batch buffers."""
    width: int
    height: int
    k: int
    key_slot: int
    iv: bytes
    pixel_offset: int = 0
    public_offset: int = 0
    private_offset: int = 0


def _align16(x: int) -> int:
    return (x + 15) & ~15


def layout(descs: Sequence[ImageDesc]) -> tuple[int, int, int]:
    """Assign packed offsets (pixels 8-aligned, fragments 16-aligned) in place; returns the
    (pixel, public, private) buffer sizes in bytes."""
    px = pub = priv = 0
    for d in descs:
        pb, vb = sizes(d.width, d.height, d.k)
        d.pixel_offset, d.public_offset, d.private_offset = px, pub, priv
        px += (d.width * d.height * 3 + 7) & ~7
        pub = _align16(pub + pb)
        priv = _align16(priv + vb)
    return px, pub, priv


# struct fds_image as a numpy record (the same 56 bytes as _lib.FdsImage)
FDS_IMAGE_DTYPE = None


def fds_image_dtype():
    global FDS_IMAGE_DTYPE
    if FDS_IMAGE_DTYPE is None:
        import numpy as np
        FDS_IMAGE_DTYPE = np.dtype([("pixel_offset", "<u8"), ("public_offset", "<u8"), ("private_offset", "<u8"),
                                    ("width", "<i4"), ("height", "<i4"), ("k", "<i4"), ("key_slot", "<i4"),
                                    ("iv", "u1", (16,))])
        assert FDS_IMAGE_DTYPE.itemsize == ctypes.sizeof(_lib.FdsImage)
    return FDS_IMAGE_DTYPE


def layout_arrays(pixel_bytes, public_bytes, private_bytes):
    """layout() over arrays of per-image sizes (numpy int64): the (pixel, public, private)
    offsets, packed as layout() packs them (pixels 8-aligned, fragments 16-aligned), and the
    three buffer sizes."""
    import numpy as np
    out = []
    for b, a in ((pixel_bytes, 7), (public_bytes, 15), (private_bytes, 15)):
        step = (np.asarray(b, dtype=np.int64) + a) & ~a
        end = np.cumsum(step)
        out.append((end - step, int(end[-1]) if len(end) else 0))
    return tuple(o for o, _ in out), tuple(t for _, t in out)


def desc_records(widths, heights, ks, key_slots, ivs, offsets):
    """The fds_image descriptors of a batch as one numpy record array: per-image fields as
    sequences, ivs as 16-byte strings, offsets as returned by layout_arrays."""
    import numpy as np
    n = len(widths)
    rec = np.zeros(n, dtype=fds_image_dtype())
    rec["pixel_offset"], rec["public_offset"], rec["private_offset"] = offsets
    rec["width"], rec["height"], rec["k"], rec["key_slot"] = widths, heights, ks, key_slots
    if n:
        rec["iv"] = np.frombuffer(b"".join(_check_key(v, "iv") for v in ivs), dtype=np.uint8).reshape(n, 16)
    return rec


def copy_many(dsts, srcs, nbytes, stream: torch.cuda.Stream | None = None) -> None:
    """fds_copy_many: copy i moves nbytes[i] bytes from address srcs[i] to address dsts[i]
    (host or device pointers as integers), all enqueued on `stream` by one call."""
    import numpy as np
    d = np.ascontiguousarray(dsts, dtype=np.uint64)
    s_ = np.ascontiguousarray(srcs, dtype=np.uint64)
    b = np.ascontiguousarray(nbytes, dtype=np.uint64)
    if not (len(d) == len(s_) == len(b)):
        raise ValueError("copy_many: dsts, srcs and nbytes differ in length")
    st = (stream or torch.cuda.current_stream()).cuda_stream
    _lib.check(_lib.load().fds_copy_many(d.ctypes.data, s_.ctypes.data, b.ctypes.data, len(d), st),
               "fds_copy_many")


def _desc_array(descs: Sequence[ImageDesc]):
    arr = (_lib.FdsImage * max(1, len(descs)))()
    for i, d in enumerate(descs):
        e = arr[i]
        e.pixel_offset, e.public_offset, e.private_offset = d.pixel_offset, d.public_offset, d.private_offset
        e.width, e.height, e.k, e.key_slot = d.width, d.height, d.k, d.key_slot
        ctypes.memmove(e.iv, _check_key(d.iv, "iv"), 16)
    return arr


def protect(pixels: torch.Tensor, public_out: torch.Tensor, private_out: torch.Tensor,
            descs: Sequence[ImageDesc]) -> None:
    """fds_protect: a batch of images in three flat device buffers (uint8)."""
    arr = _desc_array(descs)
    rc = _lib.load().fds_protect(pixels.data_ptr(), public_out.data_ptr(), private_out.data_ptr(),
                                 arr, len(descs), _stream_ptr(pixels.device))
    _lib.check(rc, "fds_protect")


def restore(public: torch.Tensor, private: torch.Tensor, pixels_out: torch.Tensor,
            descs: Sequence[ImageDesc]) -> None:
    """fds_restore: inverse of protect() for a batch."""
    arr = _desc_array(descs)
    rc = _lib.load().fds_restore(public.data_ptr(), private.data_ptr(), pixels_out.data_ptr(),
                                 arr, len(descs), _stream_ptr(pixels_out.device))
    _lib.check(rc, "fds_restore")


def debug_dct_f32(pixels: torch.Tensor) -> torch.Tensor:
    """fds_debug_dct_f32: float32 coefficients [H/8, W/8, 3, 8, 8] before rounding."""
    w, h = _image_dims(pixels)
    out = torch.empty((h // 8, w // 8, 3, 8, 8), dtype=torch.float32, device=pixels.device)
    rc = _lib.load().fds_debug_dct_f32(pixels.data_ptr(), w, h, out.data_ptr(),
                                       _stream_ptr(pixels.device))
    _lib.check(rc, "fds_debug_dct_f32")
    return out


def sizes_packed(width: int, height: int, k: int, form: int = 11) -> tuple[int, int, int]:
    """fds_sizes_packed: (packed public bytes, packed private bytes, scratch bytes)."""
    pub, priv, scr = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _lib.check(_lib.load().fds_sizes_packed(form, width, height, k, ctypes.byref(pub), ctypes.byref(priv),
                                            ctypes.byref(scr)), "fds_sizes_packed")
    return pub.value, priv.value, scr.value


def protect_image_packed(pixels: torch.Tensor, key: bytes, iv: bytes, k: int, form: int = 11,
                         scratch: torch.Tensor | None = None, public: torch.Tensor | None = None,
                         private: torch.Tensor | None = None) -> tuple[torch.Tensor, torch.Tensor]:
    """fds_protect_image_packed: (packed public bytes, packed private ciphertext) as uint8
    device tensors (11-bit or 8-bit storage); `public` / `private` are optional output buffers
    of at least the fds_sizes_packed byte counts."""
    w, h = _image_dims(pixels)
    pub_b, priv_b, scr_b = sizes_packed(w, h, k, form)
    dev = pixels.device
    pub = torch.empty(max(pub_b, 1), dtype=torch.uint8, device=dev) if public is None else public
    priv = torch.empty(max(priv_b, 16), dtype=torch.uint8, device=dev) if private is None else private
    if pub.numel() < pub_b or priv.numel() < priv_b or pub.dtype != torch.uint8 or priv.dtype != torch.uint8:
        raise ValueError("packed output buffers too small or not uint8")
    if scratch is None:
        scratch = torch.empty(scr_b, dtype=torch.uint8, device=dev)
    rc = _lib.load().fds_protect_image_packed(form, pixels.data_ptr(), w, h, k, _check_key(key, "key"),
                                              _check_key(iv, "iv"), pub.data_ptr(), priv.data_ptr(),
                                              scratch.data_ptr(), _stream_ptr(dev))
    _lib.check(rc, "fds_protect_image_packed")
    return pub[:pub_b], priv[:priv_b]


def restore_image_packed(public: torch.Tensor, private: torch.Tensor, width: int, height: int, k: int,
                         key: bytes, iv: bytes, form: int = 11,
                         scratch: torch.Tensor | None = None, out: torch.Tensor | None = None) -> torch.Tensor:
    """fds_restore_image_packed: the H x W x 3 uint8 image (into `out` when given)."""
    dev = private.device
    _, _, scr_b = sizes_packed(width, height, k, form)
    if scratch is None:
        scratch = torch.empty(scr_b, dtype=torch.uint8, device=dev)
    if out is None:
        out = torch.empty((height, width, 3), dtype=torch.uint8, device=dev)
    elif out.shape != (height, width, 3) or out.dtype != torch.uint8 or not out.is_contiguous():
        raise ValueError("out must be a contiguous H x W x 3 uint8 tensor")
    rc = _lib.load().fds_restore_image_packed(form, public.data_ptr() if public.numel() else None,
                                              private.data_ptr(), width, height, k, _check_key(key, "key"),
                                              _check_key(iv, "iv"), out.data_ptr(), scratch.data_ptr(),
                                              _stream_ptr(dev))
    _lib.check(rc, "fds_restore_image_packed")
    return out


def protect_image_host(host_pixels: torch.Tensor, dev_pixels: torch.Tensor, key: bytes, iv: bytes, k: int,
                       dev_public: torch.Tensor, dev_private: torch.Tensor, host_public: torch.Tensor,
                       host_private: torch.Tensor, strips: int = 8) -> None:
    """fds_protect_image_host: host pixels -> device -> protect -> both fragments back to the
    host, by strips with the copies overlapped (host tensors should be pinned)."""
    w, h = int(host_pixels.shape[1]), int(host_pixels.shape[0])
    for t in (host_pixels, host_public, host_private):
        if t.is_cuda or not t.is_contiguous():
            raise ValueError("host buffers must be contiguous CPU tensors")
    for t in (dev_pixels, dev_public, dev_private):
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError("device buffers must be contiguous CUDA tensors")
    rc = _lib.load().fds_protect_image_host(host_pixels.data_ptr(), dev_pixels.data_ptr(), w, h, k,
                                            _check_key(key, "key"), _check_key(iv, "iv"),
                                            dev_public.data_ptr() if dev_public.numel() else None,
                                            dev_private.data_ptr(),
                                            host_public.data_ptr() if host_public.numel() else None,
                                            host_private.data_ptr(), strips, _stream_ptr(dev_pixels.device))
    _lib.check(rc, "fds_protect_image_host")


def restore_image_host(dev_public: torch.Tensor, dev_private: torch.Tensor, dev_pixels: torch.Tensor,
                       host_pixels: torch.Tensor, key: bytes, iv: bytes, k: int, strips: int = 8) -> None:
    """fds_restore_image_host: restore on the device, pixels back to the host by strips."""
    w, h = int(host_pixels.shape[1]), int(host_pixels.shape[0])
    if host_pixels.is_cuda or not host_pixels.is_contiguous():
        raise ValueError("host_pixels must be a contiguous CPU tensor")
    rc = _lib.load().fds_restore_image_host(dev_public.data_ptr() if dev_public.numel() else None,
                                            dev_private.data_ptr(), dev_pixels.data_ptr(), host_pixels.data_ptr(),
                                            w, h, k, _check_key(key, "key"), _check_key(iv, "iv"), strips,
                                            _stream_ptr(dev_pixels.device))
    _lib.check(rc, "fds_restore_image_host")


def public_image(public: torch.Tensor, width: int, height: int, k: int,
                 out: torch.Tensor | None = None) -> torch.Tensor:
    """fds_public_image: the paper-form public fragment, an H x W x 3 uint8 image (private
    zigzag positions zero, DC 1024, exact inverse DCT, rounded and clamped)."""
    dev = public.device
    if out is None:
        out = torch.empty((height, width, 3), dtype=torch.uint8, device=dev)
    elif out.shape != (height, width, 3) or out.dtype != torch.uint8 or not out.is_contiguous():
        raise ValueError("out must be a contiguous H x W x 3 uint8 tensor")
    if public.numel() and (public.dtype != torch.int16 or not public.is_contiguous()):
        raise ValueError("public must be a contiguous int16 tensor")
    rc = _lib.load().fds_public_image(public.data_ptr() if public.numel() else None, width, height, k,
                                      out.data_ptr(), _stream_ptr(dev))
    _lib.check(rc, "fds_public_image")
    return out


def image_stats(image: torch.Tensor) -> tuple[torch.Tensor, torch.Tensor]:
    """fds_image_stats: (histogram uint64-as-int64 [3, 256], pair sums int64 [3, 3, 6]) as
    device tensors; see correlation() for r."""
    if image.dtype != torch.uint8 or image.dim() != 3 or image.shape[2] != 3 or not image.is_contiguous():
        raise ValueError("image must be a contiguous H x W x 3 uint8 tensor")
    h, w, _ = image.shape
    hist = torch.empty((3, 256), dtype=torch.int64, device=image.device)
    sums = torch.empty((3, 3, 6), dtype=torch.int64, device=image.device)
    rc = _lib.load().fds_image_stats(image.data_ptr(), w, h, hist.data_ptr(), sums.data_ptr(),
                                     _stream_ptr(image.device))
    _lib.check(rc, "fds_image_stats")
    return hist, sums


def correlation(sums) -> list:
    """Correlation coefficients r [direction][channel] (right, down, down-right) from the exact
    pair sums of image_stats (Sect. 6.6.2); None where a variance is zero."""
    s = sums.tolist() if hasattr(sums, "tolist") else sums
    out = []
    for d in range(3):
        row = []
        for c in range(3):
            n, sx, sy, sxx, syy, sxy = (int(v) for v in s[d][c])
            dx, dy = n * sxx - sx * sx, n * syy - sy * sy
            row.append((n * sxy - sx * sy) / math.sqrt(dx * dy) if dx > 0 and dy > 0 else None)
        out.append(row)
    return out


def sizes_strong(width: int, height: int, k: int) -> tuple[int, int, int]:
    """fds_sizes_strong: (public image bytes, private bytes, scratch bytes)."""
    pub, priv, scr = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _lib.check(_lib.load().fds_sizes_strong(width, height, k, ctypes.byref(pub), ctypes.byref(priv),
                                            ctypes.byref(scr)), "fds_sizes_strong")
    return pub.value, priv.value, scr.value


def protect_image_strong(pixels: torch.Tensor, key: bytes, iv: bytes, k: int,
                         scratch: torch.Tensor | None = None, public: torch.Tensor | None = None,
                         private: torch.Tensor | None = None) -> tuple[torch.Tensor, torch.Tensor]:
    """fds_protect_image_strong: (strong public image H x W x 3 uint8, Part 1 ciphertext)."""
    w, h = _image_dims(pixels)
    _, priv_b, scr_b = sizes_strong(w, h, k)
    dev = pixels.device
    if public is None:
        public = torch.empty((h, w, 3), dtype=torch.uint8, device=dev)
    if private is None:
        private = torch.empty(priv_b, dtype=torch.uint8, device=dev)
    if scratch is None:
        scratch = torch.empty(scr_b, dtype=torch.uint8, device=dev)
    if public.shape != (h, w, 3) or public.dtype != torch.uint8 or private.numel() < priv_b:
        raise ValueError("bad output buffers")
    rc = _lib.load().fds_protect_image_strong(pixels.data_ptr(), w, h, k, _check_key(key, "key"),
                                              _check_key(iv, "iv"), public.data_ptr(), private.data_ptr(),
                                              scratch.data_ptr(), _stream_ptr(dev))
    _lib.check(rc, "fds_protect_image_strong")
    return public, private[:priv_b]


def restore_image_strong(public: torch.Tensor, private: torch.Tensor, k: int, key: bytes, iv: bytes,
                         scratch: torch.Tensor | None = None, out: torch.Tensor | None = None) -> torch.Tensor:
    """fds_restore_image_strong: the H x W x 3 uint8 image from the strong public image."""
    w, h = _image_dims(public)
    _, _, scr_b = sizes_strong(w, h, k)
    dev = public.device
    if scratch is None:
        scratch = torch.empty(scr_b, dtype=torch.uint8, device=dev)
    if out is None:
        out = torch.empty((h, w, 3), dtype=torch.uint8, device=dev)
    rc = _lib.load().fds_restore_image_strong(public.data_ptr(), private.data_ptr(), w, h, k,
                                              _check_key(key, "key"), _check_key(iv, "iv"), out.data_ptr(),
                                              scratch.data_ptr(), _stream_ptr(dev))
    _lib.check(rc, "fds_restore_image_strong")
    return out


def dwt_sizes(width: int, height: int) -> tuple[int, int, int]:
    """fds_dwt_sizes: bytes of level 1, level 2 and level 3 (5, 16, 60 per 8x8 block)."""
    a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _lib.check(_lib.load().fds_dwt_sizes(width, height, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
               "fds_dwt_sizes")
    return a.value, b.value, c.value


def bytes_to_matrix(data: torch.Tensor, width: int) -> torch.Tensor:
    """Agnostic chunking (Sect. 6.9.3): a 1-D uint8 tensor as rows of `width` bytes, zero-padded
    to whole 8-row blocks (the caller keeps the original length)."""
    if width <= 0 or width % 8:
        raise ValueError("width must be a positive multiple of 8")
    n = data.numel()
    rows = -(-n // width)                   # ceil(n / width)
    rows = max(8, -(-rows // 8) * 8)        # whole 8-row blocks
    out = torch.zeros(rows * width, dtype=torch.uint8, device=data.device)
    out[:n] = data.reshape(-1)
    return out.reshape(rows, width)


def dwt_protect(data: torch.Tensor, key: bytes, iv: bytes, out: tuple | None = None):
    """fds_dwt_protect: (level 1 ciphertext, level 2 masked, level 3 masked) uint8 device
    tensors of an H x W uint8 matrix."""
    if data.dtype != torch.uint8 or data.dim() != 2 or not data.is_contiguous() or not data.is_cuda:
        raise ValueError("data must be a contiguous H x W uint8 CUDA tensor")
    h, w = data.shape
    sizes = dwt_sizes(w, h)
    if out is None:
        out = tuple(torch.empty(n, dtype=torch.uint8, device=data.device) for n in sizes)
    rc = _lib.load().fds_dwt_protect(data.data_ptr(), w, h, _check_key(key, "key"), _check_key(iv, "iv"),
                                     out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(),
                                     _stream_ptr(data.device))
    _lib.check(rc, "fds_dwt_protect")
    return out


def dwt_restore(level1: torch.Tensor, level2: torch.Tensor, level3: torch.Tensor, width: int, height: int,
                key: bytes, iv: bytes, out: torch.Tensor | None = None) -> torch.Tensor:
    """fds_dwt_restore: the H x W uint8 matrix back, exactly."""
    dev = level1.device
    if out is None:
        out = torch.empty((height, width), dtype=torch.uint8, device=dev)
    rc = _lib.load().fds_dwt_restore(level1.data_ptr(), level2.data_ptr(), level3.data_ptr(), width, height,
                                     _check_key(key, "key"), _check_key(iv, "iv"), out.data_ptr(), _stream_ptr(dev))
    _lib.check(rc, "fds_dwt_restore")
    return out


def sha512_constants() -> tuple[list[int], list[int]]:
    """fds_sha512_constants (host only): the 80 round constants and the 8 initial words."""
    kk, hh = (ctypes.c_uint64 * 80)(), (ctypes.c_uint64 * 8)()
    _lib.check(_lib.load().fds_sha512_constants(kk, hh), "fds_sha512_constants")
    return list(kk), list(hh)


def encrypt_full(data: torch.Tensor, key: bytes, iv: bytes,
                 out: torch.Tensor | None = None) -> torch.Tensor:
    """fds_encrypt_full: AES-128-CTR over the whole byte buffer (the full-encryption
    comparator); `out` may be `data` itself."""
    flat = data.reshape(-1).view(torch.uint8)
    if out is None:
        out = torch.empty_like(flat)
    dst = out.reshape(-1).view(torch.uint8)
    assert dst.numel() == flat.numel()
    rc = _lib.load().fds_encrypt_full(flat.data_ptr() if flat.numel() else None,
                                      dst.data_ptr() if dst.numel() else None, flat.numel(),
                                      _check_key(key, "key"), _check_key(iv, "iv"),
                                      _stream_ptr(data.device))
    _lib.check(rc, "fds_encrypt_full")
    return out


def tc_basis(form: str = "bf16") -> tuple[bytes, float]:
    """fds_tc_basis (host only): the tensor-core B operand bytes and the proven bound on the
    pre-rounding coefficient error ("f16_inverse": the inverse transform's table and its bound
    per unit of sum |q|)."""
    f = _lib.FDS_TC_F16_INVERSE if form == "f16_inverse" else _tc_form(form)
    n = {_lib.FDS_TC_BF16: 24576, _lib.FDS_TC_TF32: 32768, _lib.FDS_TC_F16: 24576,
         _lib.FDS_TC_F16_INVERSE: 24576}[f]
    buf = (ctypes.c_uint8 * n)()
    bound = ctypes.c_double()
    _lib.check(_lib.load().fds_tc_basis(f, buf, n, ctypes.byref(bound)), "fds_tc_basis")
    return bytes(buf), bound.value


def debug_dct_tc(pixels: torch.Tensor, form: str = "bf16") -> torch.Tensor:
    """fds_debug_dct_tc: the tensor-core form's float32 coefficients [H/8, W/8, 3, 8, 8]
    before rounding."""
    f = _tc_form(form)
    w, h = _image_dims(pixels)
    out = torch.empty((h // 8, w // 8, 3, 8, 8), dtype=torch.float32, device=pixels.device)
    rc = _lib.load().fds_debug_dct_tc(f, pixels.data_ptr(), w, h, out.data_ptr(),
                                      _stream_ptr(pixels.device))
    _lib.check(rc, "fds_debug_dct_tc")
    return out


def debug_exact_round(coords) -> list[int]:
    """fds_debug_exact_round (host in, host out): the device's exact round-half-away of V_i
    with 8 V_i = coords[i][0] + sum_j coords[i][j] cos(j pi/16), for an n x 8 integer array."""
    flat = [int(v) for row in coords for v in row]
    n = len(flat) // 8
    if len(flat) != 8 * n:
        raise ValueError("coords must be rows of 8 integers")
    cin = (ctypes.c_int32 * max(1, len(flat)))(*flat)
    out = (ctypes.c_int32 * max(1, n))()
    _lib.check(_lib.load().fds_debug_exact_round(cin, out, n), "fds_debug_exact_round")
    return [int(out[i]) for i in range(n)]


def counters(reset: bool = False) -> tuple[int, int, int]:
    """fds_counters: (exact re-decisions, 256-bit escalations among them, failures)."""
    out = (ctypes.c_uint64 * 3)()
    _lib.check(_lib.load().fds_counters(out, 1 if reset else 0), "fds_counters")
    return int(out[0]), int(out[1]), int(out[2])


def debug_set_counters(values) -> None:
    """fds_debug_set_counters: overwrite the three device counters (a test hook)."""
    arr = (ctypes.c_uint64 * 3)(*[int(v) for v in values])
    _lib.check(_lib.load().fds_debug_set_counters(arr), "fds_debug_set_counters")


def sync() -> None:
    """fds_sync on the current stream."""
    _lib.check(_lib.load().fds_sync(_stream_ptr(torch.device("cuda"))), "fds_sync")


_DIRECTIONS = {"protect": 0, "restore": 1}


class Plan:
    """fds_plan_*: a batch whose descriptors and tile schedule live on the device, run as one
    persistent launch (optionally through a CUDA graph)."""

    def __init__(self, descs: Sequence[ImageDesc] | None = None, capacity: int = 0):
        """A plan for `descs`, or (descs None) an empty reusable plan for `capacity` images."""
        h = ctypes.c_void_p()
        if descs is None:
            _lib.check(_lib.load().fds_plan_reserve(capacity, ctypes.byref(h)), "fds_plan_reserve")
            self.descs = []
        else:
            arr = _desc_array(descs)
            _lib.check(_lib.load().fds_plan_create(arr, len(descs), ctypes.byref(h)),
                       "fds_plan_create")
            self.descs = list(descs)
        self._h = h

    def update(self, descs: Sequence[ImageDesc], stream: torch.cuda.Stream | None = None) -> None:
        """fds_plan_update: replace the batch of a reusable plan (copies on `stream`)."""
        arr = _desc_array(descs)
        s = (stream or torch.cuda.current_stream()).cuda_stream
        _lib.check(_lib.load().fds_plan_update(self._h, arr, len(descs), s), "fds_plan_update")
        self.descs = list(descs)

    def update_records(self, rec, stream: torch.cuda.Stream | None = None) -> None:
        """fds_plan_update from a record array of desc_records (no ImageDesc objects)."""
        import numpy as np
        rec = np.ascontiguousarray(rec, dtype=fds_image_dtype())
        s = (stream or torch.cuda.current_stream()).cuda_stream
        ptr = ctypes.cast(rec.ctypes.data, ctypes.POINTER(_lib.FdsImage))
        _lib.check(_lib.load().fds_plan_update(self._h, ptr, len(rec), s), "fds_plan_update")
        self.descs = None

    def close(self) -> None:
        if self._h:
            _lib.load().fds_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_schedule(self, ctas_per_sm: int = 0, dynamic: bool = False,
                     largest_first: bool = False) -> None:
        """fds_plan_set_schedule: both directions (ctas_per_sm 0 = each kernel's residency)."""
        _lib.check(_lib.load().fds_plan_set_schedule(self._h, ctas_per_sm, int(dynamic),
                                                     int(largest_first)), "fds_plan_set_schedule")

    def schedule(self) -> tuple[int, int, int]:
        """(ctas_per_sm, dynamic, largest_first) of the protect direction."""
        v = [ctypes.c_int32() for _ in range(3)]
        _lib.check(_lib.load().fds_plan_get_schedule(self._h, *(ctypes.byref(x) for x in v)),
                   "fds_plan_get_schedule")
        return tuple(x.value for x in v)

    def set_direction_schedule(self, direction: str, ctas_per_sm: int = 0, dynamic: bool = False,
                               aes_pair: bool = False) -> None:
        """fds_plan_set_direction_schedule; direction "protect" or "restore"."""
        _lib.check(_lib.load().fds_plan_set_direction_schedule(
            self._h, _DIRECTIONS[direction], ctas_per_sm, int(dynamic), int(aes_pair)),
            "fds_plan_set_direction_schedule")

    def direction_schedule(self, direction: str) -> dict:
        v = [ctypes.c_int32() for _ in range(3)]
        _lib.check(_lib.load().fds_plan_get_direction_schedule(
            self._h, _DIRECTIONS[direction], *(ctypes.byref(x) for x in v)),
            "fds_plan_get_direction_schedule")
        return {"ctas_per_sm": v[0].value, "dynamic": v[1].value, "aes_pair": v[2].value}

    def autotune(self, pixels, public_out, private_out, reps: int = 3) -> tuple[int, int, int]:
        """fds_plan_autotune: protect only; returns schedule()."""
        _lib.check(_lib.load().fds_plan_autotune(self._h, pixels.data_ptr(), public_out.data_ptr(),
                                                 private_out.data_ptr(), reps,
                                                 _stream_ptr(pixels.device)), "fds_plan_autotune")
        return self.schedule()

    def schedule_json(self) -> dict:
        """fds_plan_schedule_json, parsed: size class, both directions, last candidates."""
        n = ctypes.c_int64()
        lib = _lib.load()
        _lib.check(lib.fds_plan_schedule_json(self._h, None, 0, ctypes.byref(n)), "fds_plan_schedule_json")
        buf = ctypes.create_string_buffer(n.value)
        _lib.check(lib.fds_plan_schedule_json(self._h, buf, n.value, ctypes.byref(n)),
                   "fds_plan_schedule_json")
        return json.loads(buf.value.decode())

    def tune(self, pixels, public_buf, private_buf, pixels_out, reps: int = 3,
             cache: str | os.PathLike | None = None) -> dict:
        """Per-direction schedule for this batch.  With `cache` (a JSON file of size class ->
        schedule), a stored schedule of the batch's size class is applied without timing;
        otherwise fds_plan_autotune_directions times every candidate (overwriting the three
        buffers) and the choice is stored there.  Returns schedule_json() plus "cached"."""
        store = {}
        if cache is not None and os.path.exists(cache):
            with open(cache) as f:
                store = json.load(f)
        cls = self.schedule_json()["size_class"]
        if cls in store:
            c = store[cls]
            self.set_schedule(0, False, bool(c["largest_first"]))
            for d in _DIRECTIONS:
                self.set_direction_schedule(d, c[d]["ctas_per_sm"], bool(c[d]["dynamic"]),
                                            bool(c[d]["aes_pair"]))
            return dict(self.schedule_json(), cached=True)
        _lib.check(_lib.load().fds_plan_autotune_directions(
            self._h, pixels.data_ptr(), public_buf.data_ptr(), private_buf.data_ptr(),
            pixels_out.data_ptr(), reps, _stream_ptr(pixels.device)), "fds_plan_autotune_directions")
        out = self.schedule_json()
        if cache is not None:
            store[cls] = {k: out[k] for k in ("largest_first", "protect", "restore")}
            tmp = f"{os.fspath(cache)}.tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(store, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return dict(out, cached=False)

    def protect(self, pixels, public_out, private_out, graph: bool = False) -> None:
        fn = _lib.load().fds_plan_protect_graph if graph else _lib.load().fds_plan_protect
        _lib.check(fn(self._h, pixels.data_ptr(), public_out.data_ptr(), private_out.data_ptr(),
                      _stream_ptr(pixels.device)), "fds_plan_protect")

    def restore(self, public, private, pixels_out, graph: bool = False) -> None:
        fn = _lib.load().fds_plan_restore_graph if graph else _lib.load().fds_plan_restore
        _lib.check(fn(self._h, public.data_ptr(), private.data_ptr(), pixels_out.data_ptr(),
                      _stream_ptr(pixels_out.device)), "fds_plan_restore")


def protect_batch_noalloc(pixels: torch.Tensor, public_out: torch.Tensor,
                          private_out: torch.Tensor, descs: Sequence[ImageDesc]) -> None:
    """fds_protect_batch_noalloc: the one-launch batched protect for callers that cannot
    allocate device memory; the library allocates nothing (its scratch is static device
    memory shared by all calls, so calls that overlap on the GPU must be serialised)."""
    arr = _desc_array(descs)
    rc = _lib.load().fds_protect_batch_noalloc(pixels.data_ptr(), public_out.data_ptr(),
                                               private_out.data_ptr(), arr, len(descs),
                                               _stream_ptr(pixels.device))
    _lib.check(rc, "fds_protect_batch_noalloc")
