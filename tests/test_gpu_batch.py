"""Batched form through the C ABI: one persistent launch over every tile of a batch of
uneven images (plans), with every schedule, under a CUDA graph and after autotuning, must
give the same bytes as the per-image path and as the CPU oracle."""
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


def _batch(api, sizes, ks, seed):
    descs, imgs, keys = [], [], []
    for i, ((w, h), k) in enumerate(zip(sizes, ks)):
        key = synth.make_key(seed + 1000 + i % 7)     # several images share keys
        keys.append(key)
        descs.append(api.ImageDesc(w, h, k, api.key_register(key), synth.make_iv(seed + 2000 + i)))
        imgs.append(synth.make_image(w, h, seed + i))
    npx, npub, npriv = api.layout(descs)
    px = torch.zeros(npx, dtype=torch.uint8)
    for d, img in zip(descs, imgs):
        px[d.pixel_offset: d.pixel_offset + img.size] = torch.from_numpy(img.reshape(-1))
    return descs, imgs, keys, px.to(DEV), npub, npriv


def _per_image(api, descs, px, npub, npriv):
    pub = torch.zeros(npub, dtype=torch.uint8, device=DEV)
    priv = torch.zeros(npriv, dtype=torch.uint8, device=DEV)
    api.protect(px, pub, priv, descs)
    back = torch.zeros_like(px)
    api.restore(pub, priv, back, descs)
    torch.cuda.synchronize()
    return pub.cpu().numpy(), priv.cpu().numpy(), back.cpu().numpy()


def _plan_run(plan, px, npub, npriv, graph=False, bufs=None):
    if bufs is None:
        bufs = (torch.empty(npub, dtype=torch.uint8, device=DEV),
                torch.empty(npriv, dtype=torch.uint8, device=DEV), torch.empty_like(px))
    pub, priv, back = bufs
    for b in bufs:
        b.fill_(0x5A)
    torch.cuda.synchronize()
    stream = torch.cuda.Stream() if graph else torch.cuda.current_stream()
    with torch.cuda.stream(stream):                      # graphs need a created stream
        plan.protect(px, pub, priv, graph=graph)
        plan.restore(pub, priv, back, graph=graph)
    torch.cuda.synchronize()
    return pub.cpu().numpy(), priv.cpu().numpy(), back.cpu().numpy()


def _same(descs, a, b):
    """Compare only the bytes the images own (padding between images is not written)."""
    for d in descs:
        pb, vb = ofds.sizes(d.width, d.height, d.k)
        n = d.width * d.height * 3
        assert np.array_equal(a[0][d.public_offset: d.public_offset + pb], b[0][d.public_offset: d.public_offset + pb])
        assert np.array_equal(a[1][d.private_offset: d.private_offset + vb], b[1][d.private_offset: d.private_offset + vb])
        assert np.array_equal(a[2][d.pixel_offset: d.pixel_offset + n], b[2][d.pixel_offset: d.pixel_offset + n])


SIZES = [(64, 48), (8, 8), (520, 40), (136, 72), (256, 256), (24, 16), (512, 96), (72, 520),
         (1024, 64), (8, 200)]


@pytest.mark.parametrize("ks", [[0] * len(SIZES), [5] * len(SIZES), [0, 5, 17, 63, 5, 0, 9, 1, 5, 0]])
def test_plan_matches_per_image_in_every_schedule(api, ks):
    descs, imgs, keys, px, npub, npriv = _batch(api, SIZES, ks, seed=11)
    want = _per_image(api, descs, px, npub, npriv)
    plan = api.Plan(descs)
    for lf in (0, 1):
        for dyn in (0, 1):
            for ps in (1, 2):
                plan.set_schedule(ps, bool(dyn), bool(lf))
                _same(descs, want, _plan_run(plan, px, npub, npriv))
    plan.close()
    # and the per-image path itself against the oracle, on a few images
    for i in (0, 1, 2, 4):
        d = descs[i]
        want_pub, want_priv = ofds.protect(imgs[i], keys[i], d.iv, d.k)
        pb, vb = ofds.sizes(d.width, d.height, d.k)
        assert want[0][d.public_offset: d.public_offset + pb].tobytes() == want_pub.tobytes()
        assert want[1][d.private_offset: d.private_offset + vb].tobytes() == want_priv
    for d in descs:
        api.key_release(d.key_slot)


def test_plan_graph_replay_and_autotune(api):
    rng = np.random.default_rng(3)
    sizes = [(int(w), int(h)) for w, h in synth.batch_sizes(40, 77, 64, 512)]
    descs, imgs, keys, px, npub, npriv = _batch(api, sizes, [0] * len(sizes), seed=31)
    want = _per_image(api, descs, px, npub, npriv)
    plan = api.Plan(descs)
    bufs = (torch.empty(npub, dtype=torch.uint8, device=DEV),
            torch.empty(npriv, dtype=torch.uint8, device=DEV), torch.empty_like(px))
    for _ in range(3):                                   # capture once, replay twice
        _same(descs, want, _plan_run(plan, px, npub, npriv, graph=True, bufs=bufs))
    pub = torch.empty(npub, dtype=torch.uint8, device=DEV)
    priv = torch.empty(npriv, dtype=torch.uint8, device=DEV)
    ps, dyn, lf = plan.autotune(px, pub, priv, reps=2)
    assert 1 <= ps <= 4 and dyn in (0, 1) and lf in (0, 1)
    _same(descs, want, _plan_run(plan, px, npub, npriv, graph=True, bufs=bufs))
    _same(descs, want, _plan_run(plan, px, npub, npriv, graph=False))
    plan.close()
    for d in descs:
        api.key_release(d.key_slot)
    assert rng is not None


@pytest.mark.parametrize("ks", [[5] * len(SIZES), [0, 5, 17, 63, 5, 0, 9, 1, 5, 0]])
def test_plan_direction_schedules_and_aes_lane_pairs(api, ks):
    """Every per-direction schedule (protect 1..4 CTAs/SM, restore 1..2, static or dynamic,
    one or two keystream blocks per thread) gives the per-image bytes; k = 17 and 63 tiles
    have more keystream blocks than a CTA has threads, where the paired schedule differs."""
    descs, imgs, keys, px, npub, npriv = _batch(api, SIZES, ks, seed=23)
    want = _per_image(api, descs, px, npub, npriv)
    plan = api.Plan(descs)
    for ps, rs in ((1, 1), (2, 2), (3, 1), (4, 2), (0, 0)):
        for dyn in (0, 1):
            for aes in (0, 1):
                plan.set_direction_schedule("protect", ps, bool(dyn), bool(aes))
                plan.set_direction_schedule("restore", rs, bool(1 - dyn), bool(aes))
                assert plan.direction_schedule("protect") == {"ctas_per_sm": ps, "dynamic": dyn, "aes_pair": aes}
                _same(descs, want, _plan_run(plan, px, npub, npriv))
    from paper_1512_02951_gb300 import _lib
    with pytest.raises(_lib.FdsError):
        plan.set_direction_schedule("restore", 3)
    with pytest.raises(_lib.FdsError):
        plan.set_direction_schedule("protect", 5)
    plan.close()
    for d in descs:
        api.key_release(d.key_slot)


def test_plan_tunes_both_directions_and_caches_the_choice(api, tmp_path):
    import json

    sizes = [(int(w), int(h)) for w, h in synth.batch_sizes(60, 91, 64, 512)]
    descs, imgs, keys, px, npub, npriv = _batch(api, sizes, [0] * len(sizes), seed=41)
    want = _per_image(api, descs, px, npub, npriv)
    plan = api.Plan(descs)
    bufs = (torch.empty(npub, dtype=torch.uint8, device=DEV),
            torch.empty(npriv, dtype=torch.uint8, device=DEV), torch.empty_like(px))
    cache = tmp_path / "schedules.json"
    got = plan.tune(px, *bufs, reps=2, cache=cache)
    assert got["cached"] is False
    cands = got["candidates"]
    assert len(cands) == 2 * (4 * 2 * 2 + 2 * 2 * 2)        # tile orders x protect + restore grids
    assert all(c["ms"] > 0 for c in cands)
    for d in ("protect", "restore"):                         # the kept schedule is the fastest
        best = min((c for c in cands if c["direction"] == d and c["largest_first"] == got["largest_first"]),
                   key=lambda c: c["ms"])
        assert got[d] == {k: best[k] for k in ("ctas_per_sm", "dynamic", "aes_pair")}
    _same(descs, want, _plan_run(plan, px, npub, npriv))
    stored = json.loads(cache.read_text())
    assert list(stored) == [got["size_class"]]
    plan2 = api.Plan(descs)
    again = plan2.tune(px, *bufs, cache=cache)
    assert again["cached"] is True and again["candidates"] == []
    assert {k: again[k] for k in ("largest_first", "protect", "restore")} == stored[got["size_class"]]
    _same(descs, want, _plan_run(plan2, px, npub, npriv, graph=True))
    plan.close()
    plan2.close()
    for d in descs:
        api.key_release(d.key_slot)


def test_plan_rejects_bad_descriptors(api):
    from paper_1512_02951_gb300 import _lib
    with pytest.raises(_lib.FdsError):
        api.Plan([api.ImageDesc(60, 64, 0, 0, bytes(16))])   # width not a multiple of 8
    with pytest.raises(_lib.FdsError):
        api.Plan([api.ImageDesc(64, 64, 0, 250, bytes(16))])  # key slot not registered
