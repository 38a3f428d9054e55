"""The paper-form public fragment (fds_public_image, Sect. 6.5.1 Fig. 10) and the statistics
of Sect. 6.6 (fds_image_stats) against the oracle: bit-exact images, exact integer sums."""
import numpy as np
import pytest

from oracle import fds as ofds, public as opub
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


def _gpu_public_image(api, pub, w, h, k):
    t = torch.from_numpy(np.ascontiguousarray(pub)).to(DEV) if k < 63 else torch.empty(0, dtype=torch.int16,
                                                                                         device=DEV)
    out = api.public_image(t, w, h, k)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("k", [0, 5, 17, 63])
@pytest.mark.parametrize("w,h", [(8, 8), (520, 40), (136, 72)])
def test_public_image_of_protected_images(api, k, w, h):
    # 1 .. 325 blocks: several tiles and a ragged last tile
    img = synth.make_image(w, h, w * 7 + h + k)
    pub, _ = ofds.protect(img, bytes(16), bytes(16), k)
    assert np.array_equal(_gpu_public_image(api, pub, w, h, k), opub.public_image(pub, k, w, h))


@pytest.mark.parametrize("k", [0, 5])
def test_public_image_of_arbitrary_fragments(api, k):
    # large coefficients (clamping at both ends) mixed with small ones (near ties)
    rng = np.random.default_rng(40 + k)
    pub = rng.integers(-900, 901, size=(6, 17, 3, 63 - k)).astype(np.int16)
    pub[..., 1::2] //= 37
    got = _gpu_public_image(api, pub, 136, 48, k)
    want = opub.public_image(pub, k, 136, 48)
    assert np.array_equal(got, want)
    assert (want == 0).any() and (want == 255).any()


def test_public_image_exact_ties(api):
    pub = np.zeros((3, 5, 3, 58), dtype=np.int16)
    z04, z40 = ofds.ZIGZAG.index((0, 4)), ofds.ZIGZAG.index((4, 0))
    pub[..., z04 - 6] = 4          # pixels exactly 128 +- 0.5
    pub[:, :, 1, z40 - 6] = -12    # and 128 +- 0.5 +- 1.5
    got = _gpu_public_image(api, pub, 40, 24, 5)
    assert np.array_equal(got, opub.public_image(pub, 5, 40, 24))


@pytest.mark.parametrize("k", [0, 5])
def test_public_fragment_back_from_the_public_image(api, k):
    # the paper's restore path from the public image: forward transform of the image on the
    # GPU (fds_protect_image's public output) against the oracle's
    w, h = 136, 72
    img = synth.make_image(w, h, 11 + k)
    pub, _ = ofds.protect(img, bytes(16), bytes(16), k)
    pimg = _gpu_public_image(api, pub, w, h, k)
    back, _ = api.protect_image(torch.from_numpy(pimg).to(DEV), bytes(16), bytes(16), k)
    assert np.array_equal(back.cpu().numpy(), opub.public_from_image(pimg, k))


@pytest.mark.parametrize("w,h", [(1, 1), (1, 9), (13, 7), (136, 72), (1000, 3)])
def test_stats_match_oracle(api, w, h):
    img = np.random.default_rng(w * 31 + h).integers(0, 256, size=(h, w, 3)).astype(np.uint8)
    hist, sums = api.image_stats(torch.from_numpy(img).to(DEV))
    torch.cuda.synchronize()
    assert np.array_equal(hist.cpu().numpy(), opub.histogram(img))
    assert np.array_equal(sums.cpu().numpy(), opub.pair_sums(img))


def test_stats_full_size_and_correlation(api):
    # 4096 x 4096: the whole histogram and every pair sum, exactly
    img = synth.make_image(4096, 4096, 2)
    hist, sums = api.image_stats(torch.from_numpy(img).to(DEV))
    torch.cuda.synchronize()
    assert np.array_equal(hist.cpu().numpy(), opub.histogram(img))
    s = sums.cpu().numpy()
    assert np.array_equal(s, opub.pair_sums(img))
    r_api = np.array(api.correlation(s), dtype=np.float64)
    assert np.allclose(r_api, opub.correlation(s), rtol=0, atol=1e-12)
    assert (r_api > 0.9).all()     # a smooth synthetic photograph: neighbours strongly correlated


def test_public_image_full_size_sampled(api):
    # 4096 x 4096, k = 5, in the launch configuration of the benchmark: the first and last
    # two block rows against the oracle (blocks are independent)
    w = h = 4096
    img = synth.make_image(w, h, 2)
    pub_t, _ = api.protect_image(torch.from_numpy(img).to(DEV), bytes(16), bytes(16), 5)
    got = api.public_image(pub_t, w, h, 5).cpu().numpy()
    pub = pub_t.cpu().numpy()
    for rows in (slice(0, 2), slice(h // 8 - 2, h // 8)):
        want = opub.public_image(pub[rows], 5, w, 16)
        assert np.array_equal(got[rows.start * 8: rows.start * 8 + 16], want)
