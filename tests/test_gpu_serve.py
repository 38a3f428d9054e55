"""Serving form on the GPU: requests arriving while others are on the device are batched and
overlapped, and every result is bit-identical to the same request served alone (and to the
CPU oracle)."""
import numpy as np
import pytest

from oracle import fds as ofds
from paper_1512_02951_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_02951_gb300 import api, build

    build.build()
    api.init(0)
    keys = [synth.make_key(900 + i) for i in range(64)]
    slots = [api.key_register(k) for k in keys]
    yield api, keys, slots
    for s in slots:
        api.key_release(s)


def _make(env, n, seed):
    from paper_1512_02951_gb300.serve import Request
    api, keys, slots = env
    rng = np.random.default_rng(seed)
    reqs = []
    for i, (w, h) in enumerate(synth.batch_sizes(n, seed, 64, 768)):
        k = int(rng.choice([0, 5]))
        j = int(rng.integers(0, 64))
        iv = synth.make_iv(seed * 1000 + i)
        img = synth.make_image(w, h, seed + i)
        if i % 2 == 0:
            reqs.append(Request("protect", w, h, k, slots[j], iv, pixels=img))
        else:
            pub, priv = ofds.protect(img, keys[j], iv, k)
            reqs.append(Request("restore", w, h, k, slots[j], iv, public=pub, private=priv))
    return reqs


def _clone(r):
    from paper_1512_02951_gb300.serve import Request
    return Request(r.kind, r.width, r.height, r.k, r.key_slot, r.iv, r.pixels, r.public, r.private)


def _equal(a, b):
    if isinstance(a, tuple):
        return np.array_equal(a[0], b[0]) and a[1] == b[1]
    return np.array_equal(a, b)


@pytest.mark.parametrize("budget_factor", [None, 2.5])
def test_each_result_is_the_same_alone_and_in_the_mix(env, budget_factor):
    from paper_1512_02951_gb300.serve import Server
    api, keys, slots = env
    reqs = _make(env, 48, 17)
    budget = None if budget_factor is None else int(max(r.device_bytes() for r in reqs) * budget_factor)
    mix = Server(lanes=3, max_batch=16, mem_budget=budget)
    for r in reqs:                                     # all at once: batched and overlapped
        mix.submit(r)
    got = [r.future.result(timeout=120) for r in reqs]
    stats = dict(mix.stats)
    mix.close()
    assert stats["max_batch"] > 1 and stats["batches"] < len(reqs)
    alone_srv = Server(lanes=1, max_batch=1)
    for r, g in zip(reqs, got):
        c = _clone(r)
        alone_srv.submit(c)
        assert _equal(c.future.result(timeout=60), g)
    alone_srv.close()
    for r, g in zip(reqs[:6], got[:6]):                # and the oracle
        key = keys[slots.index(r.key_slot)]
        if r.kind == "protect":
            pub, priv = ofds.protect(np.asarray(r.pixels), key, r.iv, r.k)
            assert np.array_equal(g[0], pub) and g[1] == priv
        else:
            want = ofds.restore(r.public, r.private, key, r.iv, r.k, r.width, r.height)
            assert np.array_equal(g, want)


def test_poisson_arrivals_report_latency(env):
    from paper_1512_02951_gb300.serve import Server, run_poisson
    reqs = _make(env, 40, 23)
    srv = Server(lanes=3, max_batch=16)
    out = run_poisson(srv, reqs, synth.poisson_arrivals(len(reqs), 500.0, 23))
    srv.close()
    assert out["requests"] == 40 and 0 < out["p50_ms"] <= out["p99_ms"] < 5000


def _with_outputs(r, pinned):
    """A copy of request r that brings its own output buffers (pinned or pageable)."""
    c = _clone(r)
    n, pb, vb = c.sizes()
    shapes = (pb, vb) if r.kind == "protect" else (n,)
    c.out = tuple(torch.full((b + 5,), 0xA5, dtype=torch.uint8, pin_memory=pinned) for b in shapes)
    return c


def test_caller_output_buffers_give_the_same_results(env):
    # requests that bring output buffers get their results straight from the device; in a
    # mix with requests that do not, every result equals the one served the usual way
    from paper_1512_02951_gb300.serve import Server
    reqs = _make(env, 36, 31)
    srv = Server(lanes=2, max_batch=12)
    base = [_clone(r) for r in reqs]
    for r in base:
        srv.submit(r)
    want = [r.future.result(timeout=120) for r in base]
    mixed = [(_with_outputs(r, pinned=(i % 3 != 2)) if i % 4 != 3 else _clone(r)) for i, r in enumerate(reqs)]
    for r in mixed:
        srv.submit(r)
    got = [r.future.result(timeout=120) for r in mixed]
    srv.close()
    for r, g, w in zip(mixed, got, want):
        assert _equal(g, w), (r.kind, r.width, r.height, r.k)
        if r.out is not None:                         # the result lies in the caller's buffer
            n, pb, vb = r.sizes()
            if r.kind == "protect":
                assert g[0].ctypes.data == r.out[0].data_ptr()
                assert r.out[0][pb:].eq(0xA5).all() and r.out[1][vb:].eq(0xA5).all()
            else:
                assert g.ctypes.data == r.out[0].data_ptr() and r.out[0][n:].eq(0xA5).all()


def test_request_buffers_are_checked_at_submission(env):
    from paper_1512_02951_gb300.serve import Request, Server
    srv = Server(lanes=1, max_batch=4)
    img = synth.make_image(16, 8, 3)
    with pytest.raises(ValueError):                   # input of the wrong size
        srv.submit(Request("protect", 16, 16, 0, env[2][0], synth.make_iv(1), pixels=img))
    r = Request("protect", 16, 8, 0, env[2][0], synth.make_iv(1), pixels=img)
    n, pb, vb = r.sizes()
    r.out = (torch.empty(pb, dtype=torch.uint8), torch.empty(vb - 1, dtype=torch.uint8))
    with pytest.raises(ValueError):                   # output buffer too small
        srv.submit(r)
    srv.close()


def test_copy_many_moves_every_range(env):
    # fds_copy_many on its own: host -> device, device -> host and device -> device ranges of
    # uneven sizes (0 and 1 byte included) in one call each, on a side stream
    from paper_1512_02951_gb300 import api
    rng = np.random.default_rng(5)
    sizes = [0, 1, 7, 16, 4099, 65536, 3, 1 << 20]
    src = [torch.from_numpy(rng.integers(0, 256, n, dtype=np.uint8)).pin_memory() for n in sizes]
    dev = torch.zeros(sum(sizes) + 64, dtype=torch.uint8, device="cuda")
    offs = np.concatenate(([0], np.cumsum(sizes)[:-1])).astype(np.uint64)
    s = torch.cuda.Stream()
    api.copy_many(dev.data_ptr() + offs, [t.data_ptr() for t in src], sizes, s)
    back = [torch.full((n,), 7, dtype=torch.uint8).pin_memory() for n in sizes]
    api.copy_many([t.data_ptr() for t in back], dev.data_ptr() + offs, sizes, s)
    dev2 = torch.zeros_like(dev)
    api.copy_many(dev2.data_ptr() + offs, dev.data_ptr() + offs, sizes, s)
    s.synchronize()
    for a, b in zip(src, back):
        assert torch.equal(a, b)
    assert torch.equal(dev, dev2) and int(dev[sum(sizes):].sum()) == 0
