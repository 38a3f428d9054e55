"""Strong level of protection on the GPU (fds_protect_image_strong / fds_restore_image_strong,
Sect. 6.3.2 Fig. 8) against the oracle: strong public image, Part 1 ciphertext and restored
image bit-exact."""
import numpy as np
import pytest

from oracle import strong as ostrong
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
    _api.counters(reset=True)
    yield _api
    assert _api.counters()[2] == 0, "exact-rounding consistency failure"


@pytest.mark.parametrize("k", [0, 5, 17, 54, 55, 63])
@pytest.mark.parametrize("w,h", [(8, 8), (136, 72), (520, 40)])
def test_strong_matches_oracle(api, k, w, h):
    # k = 54: Part 1 fills one SHA-512 block (110 + 17 bytes); k = 55 and up take two
    img = synth.make_image(w, h, 3 * w + h + k)
    key, iv = synth.make_key(80 + k), synth.make_iv(90 + k)
    s_img, priv = api.protect_image_strong(torch.from_numpy(img).to(DEV), key, iv, k)
    torch.cuda.synchronize()
    want_img, want_priv = ostrong.protect_strong(img, key, iv, k)
    assert np.array_equal(s_img.cpu().numpy(), want_img)
    assert priv.cpu().numpy().tobytes() == want_priv
    back = api.restore_image_strong(s_img, priv, k, key, iv).cpu().numpy()
    assert np.array_equal(back, ostrong.restore_strong(want_img, want_priv, key, iv, k))


def test_strong_full_size_sampled(api):
    # 4096 x 4096, k = 5: the strong image depends on the block alone (not on key or
    # position), so the first and last two block rows match the oracle on those rows; the Part 1
    # ciphertext equals the first level's
    w = h = 4096
    img = synth.make_image(w, h, 2)
    key, iv = synth.make_key(1), synth.make_iv(2)
    t = torch.from_numpy(img).to(DEV)
    s_img, priv = api.protect_image_strong(t, key, iv, 5)
    _, priv1 = api.protect_image(t, key, iv, 5)
    assert torch.equal(priv, priv1)
    got = s_img.cpu().numpy()
    for r0 in (0, h - 16):
        want, _ = ostrong.protect_strong(img[r0: r0 + 16], key, iv, 5)
        assert np.array_equal(got[r0: r0 + 16], want)
    back = api.restore_image_strong(s_img, priv, 5, key, iv).cpu().numpy()
    for r0 in (0, h - 16):
        want_img, want_priv = ostrong.protect_strong(img[r0: r0 + 16], key, iv, 5)
        assert np.array_equal(back[r0: r0 + 16], ostrong.restore_strong(want_img, want_priv, key, iv, 5))
