"""The full-encryption comparator (fds_encrypt_full, AES-128-CTR over a whole buffer) against
the oracle's FIPS-197 / SP 800-38A CTR, on ragged sizes, counter carries and the 4096^2
image, in place and out of place."""
import numpy as np
import pytest

from oracle import aes as oaes
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


@pytest.mark.parametrize("n", [1, 15, 16, 17, 4101, (1 << 20) + 3])
def test_matches_oracle_ctr(api, n):
    rng = np.random.default_rng(n)
    data = rng.integers(0, 256, n, dtype=np.uint8)
    key, iv = synth.make_key(50 + n % 7), synth.make_iv(60 + n % 5)
    got = api.encrypt_full(torch.from_numpy(data).to(DEV), key, iv).cpu().numpy().tobytes()
    assert got == oaes.ctr_xcrypt(key, iv, data.tobytes())


@pytest.mark.parametrize("iv", [bytes(8) + b"\xff" * 8, b"\xff" * 16, bytes(12) + b"\xff\xff\xff\xf0"])
def test_counter_carries(api, iv):
    data = np.arange(4096 * 16 + 9, dtype=np.uint32).astype(np.uint8)
    key = synth.make_key(77)
    got = api.encrypt_full(torch.from_numpy(data).to(DEV), key, iv).cpu().numpy().tobytes()
    assert got == oaes.ctr_xcrypt(key, iv, data.tobytes())


def test_in_place_and_round_trip(api):
    img = synth.make_image(1024, 520, 3)
    key, iv = synth.make_key(8), synth.make_iv(9)
    x = torch.from_numpy(img).to(DEV)
    y = x.clone()
    api.encrypt_full(y, key, iv, out=y)                  # in place
    assert y.cpu().numpy().tobytes() == oaes.ctr_xcrypt(key, iv, img.tobytes())
    z = api.encrypt_full(y, key, iv)                     # decryption is the same call
    assert torch.equal(z.reshape(x.shape), x)


def test_4096_image_sampled(api):
    img = synth.make_image(4096, 4096, 2)
    key, iv = synth.make_key(2005), synth.make_iv(3005)
    ct = api.encrypt_full(torch.from_numpy(img).to(DEV), key, iv).cpu().numpy()
    flat = img.reshape(-1)
    for off in (0, 16 * 1_000_003, flat.size - 4096):
        want = oaes.ctr_xcrypt(key, iv, flat[off: off + 4096].tobytes(), offset=off)
        assert ct[off: off + 4096].tobytes() == want
