"""The serving scheduler's host logic on the CPU: lanes are fakes that compute each batch with
the CPU oracle, so batching by kind, admission by memory, lane reuse and futures are tested
without a GPU."""
import threading
import time

import numpy as np
import pytest

from oracle import aes as oaes, fds as ofds
from paper_1512_02951_gb300 import synth

KEYS = [synth.make_key(700 + i) for i in range(4)]


class FakeLane:
    """Finishes a batch a little after launch; records what the scheduler did."""
    log = []
    lock = threading.Lock()

    def __init__(self, server_ref):
        self.server_ref = server_ref
        self.batch = None
        self.t_done = 0.0

    def busy(self):
        return self.batch is not None

    def done(self):
        return self.batch is not None and time.perf_counter() >= self.t_done

    def launch(self, batch):
        srv = self.server_ref[0]
        with FakeLane.lock:
            FakeLane.log.append((len(batch), {r.kind for r in batch}, srv.in_use))
        self.batch = batch
        self.t_done = time.perf_counter() + 0.003

    def finish(self):
        res = []
        for r in self.batch:
            key = KEYS[r.key_slot]
            if r.kind == "protect":
                res.append((r, ofds.protect(np.asarray(r.pixels), key, r.iv, r.k)))
            else:
                res.append((r, ofds.restore(r.public, r.private, key, r.iv, r.k, r.width, r.height)))
        self.batch = None
        return res


def _requests(n, seed):
    from paper_1512_02951_gb300.serve import Request
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        w, h = int(rng.integers(1, 9)) * 8, int(rng.integers(1, 9)) * 8
        k = int(rng.choice([0, 5]))
        slot = int(rng.integers(0, len(KEYS)))
        iv = synth.make_iv(seed + i)
        img = synth.make_image(w, h, seed + i)
        if rng.random() < 0.5:
            reqs.append(Request("protect", w, h, k, slot, iv, pixels=img))
        else:
            pub, priv = ofds.protect(img, KEYS[slot], iv, k)
            reqs.append(Request("restore", w, h, k, slot, iv, public=pub, private=priv))
    return reqs


@pytest.fixture(scope="module", autouse=True)
def built_library():
    from paper_1512_02951_gb300 import build
    build.build()


def test_scheduler_batches_by_kind_and_respects_memory():
    from paper_1512_02951_gb300.serve import Server
    FakeLane.log.clear()
    reqs = _requests(60, 5)
    budget = max(r.device_bytes() for r in reqs) * 3
    ref = [None]
    srv = Server(lanes=2, max_batch=8, mem_budget=budget, lane_factory=lambda i: FakeLane(ref))
    ref[0] = srv
    for r in reqs:
        srv.submit(r)
    for r in reqs:
        got = r.future.result(timeout=60)
        key = KEYS[r.key_slot]
        if r.kind == "protect":
            pub, priv = ofds.protect(np.asarray(r.pixels), key, r.iv, r.k)
            assert np.array_equal(got[0], pub) and got[1] == priv
        else:
            want = ofds.restore(r.public, r.private, key, r.iv, r.k, r.width, r.height)
            assert np.array_equal(got, want)
    srv.close()
    assert srv.in_use == 0
    assert sum(n for n, _, _ in FakeLane.log) == len(reqs)
    assert all(len(kinds) == 1 for _, kinds, _ in FakeLane.log)       # one kind per batch
    assert max(n for n, _, _ in FakeLane.log) <= 8
    assert max(u for _, _, u in FakeLane.log) <= budget                # admission by memory
    assert srv.stats["max_batch"] > 1                                   # batching happened


def test_oversized_request_is_rejected():
    from paper_1512_02951_gb300.serve import Server
    reqs = _requests(1, 9)
    ref = [None]
    srv = Server(lanes=1, mem_budget=reqs[0].device_bytes() - 1, lane_factory=lambda i: FakeLane(ref))
    ref[0] = srv
    with pytest.raises(ValueError):
        srv.submit(reqs[0])
    srv.close()


def test_restore_request_ciphertext_is_what_ctr_gives():
    # the fake lane's restore inputs are consistent with an independent CTR decryption
    reqs = [r for r in _requests(20, 3) if r.kind == "restore"]
    r = reqs[0]
    plain = oaes.ctr_xcrypt(KEYS[r.key_slot], r.iv, r.private)
    assert len(plain) == ofds.sizes(r.width, r.height, r.k)[1]


def test_vectorised_layout_and_descriptors_match_the_per_image_forms():
    # the serving lane builds a batch's offsets and fds_image records as arrays; they must be
    # byte for byte what layout() and the ctypes descriptor array give
    from paper_1512_02951_gb300 import api
    rng = np.random.default_rng(3)
    descs = [api.ImageDesc(int(rng.integers(1, 40)) * 8, int(rng.integers(1, 40)) * 8, int(rng.choice([0, 5, 63])),
                           int(rng.integers(0, 9)), bytes(rng.integers(0, 256, 16, dtype=np.uint8)))
             for _ in range(50)]
    totals = api.layout(descs)
    sz = np.array([(d.width * d.height * 3,) + tuple(api.sizes(d.width, d.height, d.k)) for d in descs])
    offs, tot = api.layout_arrays(sz[:, 0], sz[:, 1], sz[:, 2])
    assert tot == totals
    assert offs[0].tolist() == [d.pixel_offset for d in descs]
    assert offs[1].tolist() == [d.public_offset for d in descs]
    assert offs[2].tolist() == [d.private_offset for d in descs]
    rec = api.desc_records([d.width for d in descs], [d.height for d in descs], [d.k for d in descs],
                           [d.key_slot for d in descs], [d.iv for d in descs], offs)
    assert rec.tobytes() == bytes(api._desc_array(descs))


def test_copy_many_rejects_bad_arguments_on_the_host():
    import ctypes
    from paper_1512_02951_gb300 import _lib
    lib = _lib.load()
    one = (ctypes.c_uint64 * 1)(8)
    zero = (ctypes.c_uint64 * 1)(0)
    assert lib.fds_copy_many(None, None, None, 0, None) == _lib.FDS_OK          # nothing to copy
    assert lib.fds_copy_many(None, None, None, -1, None) == _lib.FDS_E_INVALID
    assert lib.fds_copy_many(None, one, one, 1, None) == _lib.FDS_E_INVALID     # null array
    assert lib.fds_copy_many(zero, one, one, 1, None) == _lib.FDS_E_INVALID     # null address
    assert b"null address" in lib.fds_last_error()
    assert lib.fds_copy_many(zero, zero, zero, 1, None) == _lib.FDS_OK          # empty copies are skipped


def test_buffer_checks_and_result_views_on_the_host():
    # the host side of caller output buffers and of the lane's result builders, on CPU tensors:
    # inputs of the wrong size and output buffers that are too small are rejected; results are
    # arrays over the caller's buffers, or views into one copy of the lane's buffers per batch
    import torch
    from paper_1512_02951_gb300 import api
    from paper_1512_02951_gb300.serve import Request, _BatchCopy, _check_buffers, _result_in, _result_of
    img = synth.make_image(16, 8, 1)
    r = Request("protect", 16, 8, 5, 0, synth.make_iv(1), pixels=img)
    _check_buffers(r)
    with pytest.raises(ValueError):
        _check_buffers(Request("protect", 16, 16, 5, 0, synth.make_iv(1), pixels=img))
    n, pb, vb = r.sizes()
    assert (n, pb, vb) == (16 * 8 * 3, 2 * 6 * 58, 2 * 6 * 6)
    r.out = (torch.arange(pb + 4, dtype=torch.int64).to(torch.uint8), torch.zeros(vb - 1, dtype=torch.uint8))
    with pytest.raises(ValueError):
        _check_buffers(r)
    r.out = (r.out[0], torch.arange(vb, dtype=torch.uint8))
    _check_buffers(r)
    pub, priv = _result_in(r)
    assert pub.shape == (1, 2, 3, 58) and pub.dtype == np.int16
    assert pub.ctypes.data == r.out[0].data_ptr() and priv == bytes(range(vb))
    rr = Request("restore", 16, 8, 5, 0, synth.make_iv(1), public=np.zeros(pb // 2, np.int16), private=bytes(vb))
    _check_buffers(rr)
    with pytest.raises(ValueError):
        _check_buffers(Request("restore", 16, 8, 5, 0, synth.make_iv(1), public=np.zeros(pb, np.int16),
                               private=bytes(vb)))
    # builders: two restore requests in one batch, results as views into one copy
    (offs, (npx, _, _)) = api.layout_arrays(np.array([n, n]), np.array([pb, pb]), np.array([vb, vb]))
    lane_px = torch.from_numpy(np.random.default_rng(0).integers(0, 256, npx, dtype=np.uint8))
    bc = _BatchCopy([lane_px, None], [npx, 0])
    got = [_result_of(rr, (int(offs[0][i]), int(offs[1][i]), int(offs[2][i])), bc) for i in range(2)]
    for i, g in enumerate(got):
        assert g.shape == (8, 16, 3)
        assert np.array_equal(g.reshape(-1), lane_px.numpy()[offs[0][i]: offs[0][i] + n])
    before = [g.copy() for g in got]
    lane_px.zero_()                       # the lane reuses its buffer: the results stay as they were
    assert all(np.array_equal(g, b) for g, b in zip(got, before)) and before[0].any()
