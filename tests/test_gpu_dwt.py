"""The DWT scheme on the GPU (fds_dwt_protect / fds_dwt_restore, Sect. 6.8-6.12, Fig. 18)
against the oracle: the three level streams byte for byte, and restore exact."""
import numpy as np
import pytest

from oracle import dwt as odwt
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


def _check(api, m, key, iv):
    h, w = m.shape
    l1, l2, l3 = api.dwt_protect(torch.from_numpy(np.ascontiguousarray(m)).to(DEV), key, iv)
    torch.cuda.synchronize()
    w1, w2, w3 = odwt.protect(m, key, iv)
    assert l1.cpu().numpy().tobytes() == w1
    assert l2.cpu().numpy().tobytes() == w2
    assert l3.cpu().numpy().tobytes() == w3
    back = api.dwt_restore(l1, l2, l3, w, h, key, iv).cpu().numpy()
    assert np.array_equal(back, m)


@pytest.mark.parametrize("w,h", [(8, 8), (64, 40), (136, 72), (1032, 136)])
def test_random_matrices(api, w, h):
    # 1 .. 2193 blocks: partial CTAs of 128 blocks, level-1 keystream blocks across blocks
    rng = np.random.default_rng(w + h)
    m = rng.integers(0, 256, size=(h, w), dtype=np.uint8)
    _check(api, m, synth.make_key(w), synth.make_iv(h))


def test_structured_matrices(api):
    key, iv = synth.make_key(5), synth.make_iv(6)
    yy, xx = np.mgrid[0:64, 0:64]
    cases = [np.full((64, 64), 200), (xx * 4) % 256, ((xx + yy) % 2) * 255, ((xx // 2 + yy // 3) % 2) * 255,
             np.where((xx * 7 + yy * 13) % 5 == 0, 255, 0), synth.make_image(64, 64, 9)[..., 1]]
    for m in cases:
        _check(api, np.asarray(m, dtype=np.uint8), key, iv)
    rng = np.random.default_rng(11)                       # blocks of extremes: the widest fields
    _check(api, (rng.integers(0, 2, size=(128, 128)) * 255).astype(np.uint8), key, iv)


def test_arbitrary_bytes_chunked(api):
    rng = np.random.default_rng(12)
    raw = rng.integers(0, 256, size=100_003, dtype=np.uint8)
    m = api.bytes_to_matrix(torch.from_numpy(raw).to(DEV), 512)
    want = odwt.to_matrix(raw.tobytes(), 512)
    assert np.array_equal(m.cpu().numpy(), want)
    _check(api, want, synth.make_key(13), synth.make_iv(14))


def test_full_size_grey_image(api):
    # a 4096 x 4096 matrix (262,144 blocks): the first two block rows byte for byte against the
    # oracle (same block indices and keystream offsets), the whole restore exact
    img = synth.make_image(4096, 4096, 2)[..., 0].copy()
    key, iv = synth.make_key(1), synth.make_iv(2)
    l1, l2, l3 = api.dwt_protect(torch.from_numpy(img).to(DEV), key, iv)
    w1, w2, w3 = odwt.protect(img[:16], key, iv)
    nb = 2 * 512
    assert l1.cpu().numpy()[: 5 * nb].tobytes() == w1
    assert l2.cpu().numpy()[: 16 * nb].tobytes() == w2
    assert l3.cpu().numpy()[: 60 * nb].tobytes() == w3
    back = api.dwt_restore(l1, l2, l3, 4096, 4096, key, iv)
    assert np.array_equal(back.cpu().numpy(), img)
