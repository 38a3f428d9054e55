"""The allocation-free batch protect (fds_protect_batch_noalloc), called through the C ABI,
must give exactly the bytes of the plan-based batched protect, on two calls in a row (the
second call finds the first call's descriptors in the shared scratch area and must not be
affected by them), over batches that take many descriptor chunks and at the largest batch it
accepts, and without changing the device's free memory.  This file is collected last on
purpose."""
import ctypes

import numpy as np
import pytest

from oracle import fds as ofds
from paper_1512_02951_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _batch(api, specs, seed):
    descs, imgs = [], []
    for i, (w, h, k) in enumerate(specs):
        slot = api.key_register(synth.make_key(seed + 10 * i))
        descs.append(api.ImageDesc(w, h, k, slot, synth.make_iv(seed + 10 * i + 1)))
        imgs.append(synth.make_image(w, h, seed + i))
    npx, npub, npriv = api.layout(descs)
    px = torch.zeros(npx, dtype=torch.uint8)
    for d, img in zip(descs, imgs):
        px[d.pixel_offset: d.pixel_offset + img.size] = torch.from_numpy(img.reshape(-1))
    return descs, imgs, px.to(DEV), npub, npriv


def _owned(descs, pub, priv):
    out = []
    for d in descs:
        pb, vb = ofds.sizes(d.width, d.height, d.k)
        out.append((pub[d.public_offset: d.public_offset + pb].tobytes(),
                    priv[d.private_offset: d.private_offset + vb].tobytes()))
    return out


def test_noalloc_matches_plan_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_02951_gb300 import api, build

    build.build()
    api.init(0)
    batches = [
        [(64, 48, 0), (520, 40, 5), (8, 8, 63), (256, 256, 0), (136, 72, 17), (24, 16, 5)],
        [(72, 520, 0), (8, 200, 0), (512, 96, 0)],      # smaller: stale entries must not leak in
    ]
    for bi, specs in enumerate(batches):
        descs, imgs, px, npub, npriv = _batch(api, specs, seed=400 + 100 * bi)
        want_pub = torch.zeros(npub, dtype=torch.uint8, device=DEV)
        want_priv = torch.zeros(npriv, dtype=torch.uint8, device=DEV)
        plan = api.Plan(descs)
        plan.protect(px, want_pub, want_priv)
        plan.close()
        got_pub = torch.full((npub,), 0x77, dtype=torch.uint8, device=DEV)
        got_priv = torch.full((npriv,), 0x77, dtype=torch.uint8, device=DEV)
        api.protect_batch_noalloc(px, got_pub, got_priv, descs)
        torch.cuda.synchronize()
        want = _owned(descs, want_pub.cpu().numpy(), want_priv.cpu().numpy())
        assert _owned(descs, got_pub.cpu().numpy(), got_priv.cpu().numpy()) == want
        # and the plan path is the oracle's, for one image of the batch
        d, img = descs[0], imgs[0]
        o_pub, o_priv = ofds.protect(img, synth.make_key(400 + 100 * bi), d.iv, d.k)
        assert want[0] == (o_pub.tobytes(), o_priv)
        for dd in descs:
            api.key_release(dd.key_slot)


def _noalloc_vs_plan(api, descs, px, npub, npriv):
    want_pub = torch.zeros(npub, dtype=torch.uint8, device=DEV)
    want_priv = torch.zeros(npriv, dtype=torch.uint8, device=DEV)
    plan = api.Plan(descs)
    plan.protect(px, want_pub, want_priv)
    plan.close()
    got_pub = torch.full((npub,), 0x77, dtype=torch.uint8, device=DEV)
    got_priv = torch.full((npriv,), 0x77, dtype=torch.uint8, device=DEV)
    torch.cuda.synchronize()
    api.protect_batch_noalloc(px, got_pub, got_priv, descs)      # warm: nothing loads lazily below
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    got_pub.fill_(0x55)
    got_priv.fill_(0x55)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    api.protect_batch_noalloc(px, got_pub, got_priv, descs)
    torch.cuda.synchronize()
    free2 = torch.cuda.mem_get_info()[0]
    assert free0 == free1 == free2, (free0, free1, free2)           # the call allocated nothing
    assert _owned(descs, got_pub.cpu().numpy(), got_priv.cpu().numpy()) == \
        _owned(descs, want_pub.cpu().numpy(), want_priv.cpu().numpy())


def test_noalloc_many_chunks_and_the_maximum_batch():
    # descriptors go up in chunks of 64: 300 images take five chunks, the largest batch 64
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_02951_gb300 import api, build

    build.build()
    api.init(0)
    slot = api.key_register(synth.make_key(808))
    for n, size in ((300, None), (api._lib.FDS_NOALLOC_MAX_IMAGES, (8, 8))):
        sizes = synth.batch_sizes(n, 90 + n, 8, 96) if size is None else [size] * n
        descs = [api.ImageDesc(w, h, (i % 7) if size is None else 5, slot, synth.make_iv(5000 + i))
                 for i, (w, h) in enumerate(sizes)]
        npx, npub, npriv = api.layout(descs)
        rng = np.random.default_rng(n)
        px = torch.from_numpy(rng.integers(0, 256, npx, dtype=np.uint8)).to(DEV)
        _noalloc_vs_plan(api, descs, px, npub, npriv)
    api.key_release(slot)


def test_noalloc_rejects_oversized_batches_on_the_host():
    from paper_1512_02951_gb300 import _lib, build

    build.build()
    lib = _lib.load()
    arr = (_lib.FdsImage * 1)()
    assert lib.fds_protect_batch_noalloc(None, None, None, arr, _lib.FDS_NOALLOC_MAX_IMAGES + 1,
                                         None) == _lib.FDS_E_INVALID
    assert b"4096" in lib.fds_last_error()
    assert lib.fds_protect_batch_noalloc(None, None, None, arr, 0, None) == _lib.FDS_E_INVALID
    assert ctypes.sizeof(arr) == 56
