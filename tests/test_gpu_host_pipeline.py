"""Protect / restore with host buffers (fds_protect_image_host / fds_restore_image_host): the
strip pipeline gives the same bytes as the device entry points, on both sides of the copies."""
import numpy as np
import pytest

from oracle import fds as ofds
from paper_1512_02951_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_02951_gb300 import api as _api, build

    build.build()
    _api.init(0)
    return _api


def _run(api, img, k, strips, pinned=True):
    h, w, _ = img.shape
    key, iv = synth.make_key(w + k), synth.make_iv(h + strips)
    pub_b, priv_b = api.sizes(w, h, k)
    host_px = torch.from_numpy(img).pin_memory() if pinned else torch.from_numpy(img.copy())
    dev_px = torch.empty((h, w, 3), dtype=torch.uint8, device=DEV)
    dev_pub = torch.empty(pub_b // 2, dtype=torch.int16, device=DEV)
    dev_priv = torch.empty(max(priv_b, 16), dtype=torch.uint8, device=DEV)
    host_pub = torch.empty(pub_b // 2, dtype=torch.int16)
    host_priv = torch.empty(priv_b, dtype=torch.uint8)
    if pinned:
        host_pub, host_priv = host_pub.pin_memory(), host_priv.pin_memory()
    api.protect_image_host(host_px, dev_px, key, iv, k, dev_pub, dev_priv, host_pub, host_priv, strips)
    out_dev = torch.empty_like(dev_px)
    host_out = torch.empty((h, w, 3), dtype=torch.uint8)
    if pinned:
        host_out = host_out.pin_memory()
    api.restore_image_host(dev_pub, dev_priv, out_dev, host_out, key, iv, k, strips)
    torch.cuda.current_stream().synchronize()      # the caller's stream covers every copy
    want_pub, want_priv = api.protect_image(torch.from_numpy(img).to(DEV), key, iv, k)
    want_back = api.restore_image(want_pub, want_priv, w, h, k, key, iv)
    torch.cuda.synchronize()
    assert np.array_equal(host_pub.numpy(), want_pub.reshape(-1).cpu().numpy())
    assert host_priv.numpy().tobytes() == want_priv.cpu().numpy().tobytes()[:priv_b]
    assert torch.equal(dev_pub, want_pub.reshape(-1)) and np.array_equal(host_out.numpy(), want_back.cpu().numpy())
    return host_pub.numpy(), host_priv.numpy().tobytes(), host_out.numpy(), key, iv


@pytest.mark.parametrize("k", [0, 5, 17, 63])
@pytest.mark.parametrize("strips", [1, 2, 5])
def test_strips_match_device_entry_points(api, k, strips):
    # 17 block rows: strips of 8, 8, 1 rows (or one strip), so a strip ends mid-image
    _run(api, synth.make_image(136, 136, 3 * k + strips), k, strips)


def test_against_the_oracle_and_pageable_memory(api):
    img = synth.make_image(72, 200, 5)
    pub, priv, back, key, iv = _run(api, img, 5, 3, pinned=False)
    want_pub, want_priv = ofds.protect(img, key, iv, 5)
    assert np.array_equal(pub, want_pub.reshape(-1)) and priv == want_priv
    assert np.array_equal(back, ofds.restore(want_pub, want_priv, key, iv, 5, 72, 200))


def test_full_size(api):
    _run(api, synth.make_image(4096, 4096, 2), 5, 8)


def test_two_streams_in_flight(api):
    # images alternating over two streams, each with its own buffers and its own copy streams:
    # every call's copies still end before its stream goes on, whatever runs on the other
    h, w, k = 512, 384, 5
    pub_b, priv_b = api.sizes(w, h, k)
    imgs = [synth.make_image(w, h, 40 + i) for i in range(6)]
    keys = [(synth.make_key(50 + i), synth.make_iv(60 + i)) for i in range(6)]
    lanes = []
    for _ in range(2):
        lanes.append(dict(
            s=torch.cuda.Stream(DEV), px=torch.empty((h, w, 3), dtype=torch.uint8, device=DEV),
            pub=torch.empty(pub_b // 2, dtype=torch.int16, device=DEV),
            priv=torch.empty(priv_b, dtype=torch.uint8, device=DEV),
            out=torch.empty((h, w, 3), dtype=torch.uint8, device=DEV)))
    host_in = [torch.from_numpy(m).pin_memory() for m in imgs]
    host_pub = [torch.empty(pub_b // 2, dtype=torch.int16).pin_memory() for _ in imgs]
    host_priv = [torch.empty(priv_b, dtype=torch.uint8).pin_memory() for _ in imgs]
    host_out = [torch.empty((h, w, 3), dtype=torch.uint8).pin_memory() for _ in imgs]
    torch.cuda.synchronize()
    for i in range(len(imgs)):
        ln = lanes[i % 2]
        key, iv = keys[i]
        with torch.cuda.stream(ln["s"]):
            api.protect_image_host(host_in[i], ln["px"], key, iv, k, ln["pub"], ln["priv"],
                                   host_pub[i], host_priv[i], 2)
            api.restore_image_host(ln["pub"], ln["priv"], ln["out"], host_out[i], key, iv, k, 2)
    torch.cuda.synchronize()
    for i, img in enumerate(imgs):
        key, iv = keys[i]
        want_pub, want_priv = api.protect_image(torch.from_numpy(img).to(DEV), key, iv, k)
        want_back = api.restore_image(want_pub, want_priv, w, h, k, key, iv)
        assert np.array_equal(host_pub[i].numpy(), want_pub.reshape(-1).cpu().numpy()), i
        assert host_priv[i].numpy().tobytes() == want_priv.cpu().numpy().tobytes(), i
        assert np.array_equal(host_out[i].numpy(), want_back.cpu().numpy()), i


def test_more_streams_than_copy_lanes(api):
    # 20 caller streams: 16 get their own copy streams, the rest share one pair; every call's
    # results are still complete when its stream is
    h, w, k = 64, 128, 5
    pub_b, priv_b = api.sizes(w, h, k)
    img = synth.make_image(w, h, 77)
    key, iv = synth.make_key(78), synth.make_iv(79)
    want_pub, want_priv = api.protect_image(torch.from_numpy(img).to(DEV), key, iv, k)
    want_back = api.restore_image(want_pub, want_priv, w, h, k, key, iv).cpu().numpy()
    host_in = torch.from_numpy(img).pin_memory()
    runs = []
    for _ in range(20):
        s = torch.cuda.Stream(DEV)
        r = dict(s=s, px=torch.empty((h, w, 3), dtype=torch.uint8, device=DEV),
                 pub=torch.empty(pub_b // 2, dtype=torch.int16, device=DEV),
                 priv=torch.empty(priv_b, dtype=torch.uint8, device=DEV),
                 out=torch.empty((h, w, 3), dtype=torch.uint8, device=DEV),
                 hpub=torch.empty(pub_b // 2, dtype=torch.int16).pin_memory(),
                 hpriv=torch.empty(priv_b, dtype=torch.uint8).pin_memory(),
                 hout=torch.empty((h, w, 3), dtype=torch.uint8).pin_memory())
        runs.append(r)
    torch.cuda.synchronize()
    for r in runs:
        with torch.cuda.stream(r["s"]):
            api.protect_image_host(host_in, r["px"], key, iv, k, r["pub"], r["priv"], r["hpub"], r["hpriv"], 2)
            api.restore_image_host(r["pub"], r["priv"], r["out"], r["hout"], key, iv, k, 2)
    for r in runs:
        r["s"].synchronize()                       # each stream alone covers its call's copies
        assert np.array_equal(r["hpub"].numpy(), want_pub.reshape(-1).cpu().numpy())
        assert r["hpriv"].numpy().tobytes() == want_priv.cpu().numpy().tobytes()
        assert np.array_equal(r["hout"].numpy(), want_back)
