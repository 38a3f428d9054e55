"""Tensor-core precision form (BF16 three-limb and TF32 two-limb basis split, tcgen05 MMA):
bit-exact with the CPU oracle and with the float32 CUDA-core path, and its pre-rounding
coefficients within the proven bound of the float64 DCT-II (Sect. 6.4.2, 6.4.3)."""
import numpy as np
import pytest

from oracle import dct as odct, fds as ofds
from paper_1512_02951_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
FORMS = ["bf16", "tf32", "f16"]
F16_K = {0, 5}                   # selections the f16 (warp-specialised) form is built for


def _skip_unsupported(form, k):
    if form == "f16" and k not in F16_K:
        pytest.skip("selection not instantiated for the f16 form")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_02951_gb300 import api as _api, build

    build.build()
    _api.init(0)
    _api.counters(reset=True)
    yield _api
    assert _api.counters()[2] == 0, "exact-rounding consistency failure or tensor-core timeout"


def _tc_protect(api, img, key, iv, k, form):
    pub, priv = api.protect_image_tc(torch.from_numpy(np.ascontiguousarray(img)).to(DEV), key, iv, k, form)
    torch.cuda.synchronize()
    return pub.cpu().numpy(), priv.cpu().numpy().tobytes()


def _check(api, img, k, form, seed=0):
    key, iv = synth.make_key(300 + seed), synth.make_iv(400 + seed)
    pub, priv = _tc_protect(api, img, key, iv, k, form)
    want_pub, want_priv = ofds.protect(img, key, iv, k)
    bad = np.argwhere(pub != want_pub)
    assert bad.size == 0, f"{form}: {len(bad)} public mismatches, first {bad[:5].tolist()}"
    assert priv == want_priv, f"{form}: private ciphertext differs"


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("w,h", [(8, 8), (16, 8), (64, 64), (136, 72), (520, 40)])
@pytest.mark.parametrize("k", [0, 5, 63])
def test_tc_small_and_ragged_images(api, form, w, h, k):
    _skip_unsupported(form, k)
    # 3 .. 975 channel-blocks: one partial tile, and several 128-channel-block tiles that
    # straddle pixel blocks and block rows, with a ragged last tile
    _check(api, synth.make_image(w, h, w * 5 + h), k, form, seed=w + h + k)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("k", [0, 5, 17])
def test_tc_512_generator_image(api, form, k):
    _skip_unsupported(form, k)
    _check(api, synth.make_image(512, 512, 1), k, form, seed=k)


@pytest.mark.parametrize("form", FORMS)
def test_tc_adversarial_blocks_and_fallbacks(api, form):
    from test_gpu_parity import _adversarial_image
    api.counters(reset=True)
    _check(api, _adversarial_image(), 5, form, seed=7)
    redecided, escalated, fail = api.counters()
    assert redecided > 0 and fail == 0 and escalated <= redecided


@pytest.mark.parametrize("form", FORMS)
def test_tc_coefficients_within_proven_bound(api, form):
    from test_gpu_parity import _adversarial_image
    _, bound = api.tc_basis(form)
    for img in (synth.make_image(256, 128, 5), _adversarial_image()):
        got = api.debug_dct_tc(torch.from_numpy(img).to(DEV), form).cpu().numpy().astype(np.float64)
        want = odct.dct2(odct.image_to_blocks(img))
        err = np.abs(got - want)
        assert err.max() <= bound, (err.max(), bound)
        for u in (0, 4):                                # rational coefficients are exact:
            for v in (0, 4):                            # 8 F is the integer sum +-p
                assert np.array_equal(got[..., u, v] * 8, np.round(want[..., u, v] * 8))


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("k", [0, 5])
def test_tc_4096_equals_float32_path_and_oracle_strips(api, form, k):
    from test_gpu_parity import _strip_oracle
    img = synth.make_image(4096, 4096, 2)
    key, iv = synth.make_key(2000 + k), synth.make_iv(3000 + k)
    x = torch.from_numpy(img).to(DEV)
    pub_tc, priv_tc = api.protect_image_tc(x, key, iv, k, form)
    pub_f, priv_f = api.protect_image(x, key, iv, k)
    torch.cuda.synchronize()
    assert torch.equal(pub_tc, pub_f) and torch.equal(priv_tc, priv_f)
    pub, priv = pub_tc.cpu().numpy(), priv_tc.cpu().numpy().tobytes()
    for rows in [(0, 1), (256, 257), (511, 512)]:
        want_pub, off, want_ct = _strip_oracle(img, key, iv, k, rows)
        assert np.array_equal(pub[rows[0]: rows[1]], want_pub)
        assert priv[off: off + len(want_ct)] == want_ct


@pytest.mark.parametrize("form", FORMS)
def test_tc_queue_overflow(api, form):
    # blocks with exact ties at several irrational positions fill every tile's near-tie queue
    from oracle import exact
    rng = np.random.default_rng(77)
    cand = rng.integers(0, 3, (400000, 8, 8))
    n = np.einsum("myx,yxj->mj", cand, exact.K[2, 2])
    hit = np.nonzero((n[:, 1:] == 0).all(axis=1) & (n[:, 0] % 8 == 4))[0]
    best, best_n = None, 0
    for i in hit[:200]:
        f = odct.dct2(cand[i])
        cnt = int((np.abs(f - np.floor(f) - 0.5) < 1e-9).sum())
        if cnt > best_n:
            best, best_n = cand[i], cnt
    assert best_n >= 2
    blocks = np.broadcast_to(best.astype(np.uint8), (8, 64, 3, 8, 8))
    img = odct.blocks_to_image(np.ascontiguousarray(blocks))
    api.counters(reset=True)
    _check(api, img, 5, form, seed=12)
    assert api.counters()[0] > 8 * 64 * 3 * best_n // 2
