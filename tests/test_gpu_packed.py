"""Bit-packed storage on the GPU (fds_protect_image_packed / fds_restore_image_packed)
against the oracle's packed storage (Sect. 6.4.3, Table 5), byte for byte."""
import numpy as np
import pytest

from oracle import pack
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


def _edges(w, h):
    yy, xx = np.mgrid[0:h, 0:w]
    img = np.stack([((yy // 2 + xx // 2) % 2) * 255, (xx % 8 < 4) * 255, ((yy + xx) % 3) * 120], axis=-1)
    return img.astype(np.uint8)


def _check(api, img, k, form, seed):
    h, w, _ = img.shape
    key, iv = synth.make_key(500 + seed), synth.make_iv(600 + seed)
    pub, priv = api.protect_image_packed(torch.from_numpy(np.ascontiguousarray(img)).to(DEV), key, iv, k, form)
    torch.cuda.synchronize()
    want_pub, want_priv = pack.protect_packed(img, key, iv, k, form)
    assert pub.cpu().numpy().tobytes() == want_pub
    assert priv.cpu().numpy().tobytes() == want_priv
    back = api.restore_image_packed(pub, priv, w, h, k, key, iv, form).cpu().numpy()
    assert np.array_equal(back, pack.restore_packed(want_pub, want_priv, key, iv, k, form, w, h))


@pytest.mark.parametrize("form", [11, 8])
@pytest.mark.parametrize("w,h", [(8, 8), (64, 48), (520, 40), (136, 72)])
@pytest.mark.parametrize("k", [0, 5, 17, 63])
def test_packed_matches_oracle(api, form, w, h, k):
    # 3 .. 975 channel-blocks: partial groups of eight, k = 63 (no public fragment)
    _check(api, synth.make_image(w, h, w + h + k), k, form, seed=w + k)


@pytest.mark.parametrize("form", [11, 8])
def test_packed_high_contrast_and_512(api, form):
    _check(api, _edges(64, 48), 5, form, seed=1)          # AC up to 924: 8-bit storage saturates
    _check(api, synth.make_image(512, 512, 1), 5, form, seed=2)


@pytest.mark.parametrize("form", [11, 8])
@pytest.mark.parametrize("offset", [1, 2, 3, 4, 8])
def test_packed_public_at_any_alignment(api, form, offset):
    # the packed public fragment may start at any byte; the result is the same bytes
    w, h, k = 136, 72, 5
    img = synth.make_image(w, h, 77)
    key, iv = synth.make_key(71), synth.make_iv(72)
    pub_b, priv_b, _ = api.sizes_packed(w, h, k, form)
    buf = torch.zeros(pub_b + 8, dtype=torch.uint8, device=DEV)
    pub = buf[offset:offset + pub_b]
    api.protect_image_packed(torch.from_numpy(img).to(DEV), key, iv, k, form, public=pub,
                             private=torch.empty(priv_b, dtype=torch.uint8, device=DEV))
    want_pub, want_priv = pack.protect_packed(img, key, iv, k, form)
    got = buf.cpu().numpy()
    assert got[offset:offset + pub_b].tobytes() == want_pub
    assert not got[:offset].any() and not got[offset + pub_b:].any()      # nothing written outside
    priv = torch.from_numpy(np.frombuffer(want_priv, dtype=np.uint8).copy()).to(DEV)
    back = api.restore_image_packed(pub, priv, w, h, k, key, iv, form).cpu().numpy()
    assert np.array_equal(back, pack.restore_packed(want_pub, want_priv, key, iv, k, form, w, h))
