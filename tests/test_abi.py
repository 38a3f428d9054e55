"""The C-ABI library: it builds, loads, exports every symbol of include/fds.h, and its host-side
logic (sizes, argument checks, key registry) behaves without a GPU."""
import ctypes
import os
import re

import pytest

from conftest import ROOT
from oracle import exact, fds as ofds


@pytest.fixture(scope="module")
def lib():
    from paper_1512_02951_gb300 import _lib, build

    build.build()
    return _lib.load()


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "fds.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(fds_\w+)\s*\(", src, flags=re.M)))


def test_every_declared_symbol_is_exported(lib):
    from paper_1512_02951_gb300 import _lib

    names = _declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_lib.SIGNATURES), "binding and header disagree"


def test_struct_layout_matches_header():
    from paper_1512_02951_gb300 import _lib

    assert ctypes.sizeof(_lib.FdsImage) == 56
    assert _lib.FdsImage.iv.offset == 40


@pytest.mark.parametrize("w,h,k", [(512, 512, 0), (4096, 4096, 5), (64, 8, 63), (8, 8, 17)])
def test_sizes_match_oracle(lib, w, h, k):
    pub, priv = ctypes.c_uint64(), ctypes.c_uint64()
    assert lib.fds_sizes(w, h, k, ctypes.byref(pub), ctypes.byref(priv)) == 0
    assert (pub.value, priv.value) == ofds.sizes(w, h, k)


@pytest.mark.parametrize("w,h,k", [(100, 64, 0), (64, 0, 0), (-8, 64, 0), (64, 64, 64), (64, 64, -1)])
def test_invalid_arguments_are_rejected_on_the_host(lib, w, h, k):
    pub, priv = ctypes.c_uint64(), ctypes.c_uint64()
    assert lib.fds_sizes(w, h, k, ctypes.byref(pub), ctypes.byref(priv)) == -1
    assert lib.fds_last_error()
    key = bytes(16)
    rc = lib.fds_protect_image(None, w, h, k, key, key, None, None, None)
    assert rc == -1


def test_null_and_misaligned_pointers_are_rejected(lib):
    key = bytes(16)
    assert lib.fds_protect_image(None, 64, 64, 0, key, key, 16, 16, None) == -1
    assert lib.fds_protect_image(8, 64, 64, 0, key, key, 24, 16, None) == -1   # public not 16-aligned
    assert b"aligned" in lib.fds_last_error()


def test_key_registry(lib):
    slots = []
    slot = ctypes.c_int32()
    for _ in range(256):
        assert lib.fds_key_register(bytes(range(16)), ctypes.byref(slot)) == 0
        slots.append(slot.value)
    assert sorted(slots) == list(range(256))
    assert lib.fds_key_register(bytes(16), ctypes.byref(slot)) == -6          # all slots taken
    for s in slots:
        assert lib.fds_key_release(s) == 0
    assert lib.fds_key_release(3) == -2                                        # already free


def test_device_cosine_constants_agree_with_the_oracle():
    # the CUDA path's 256-bit cosines come from a Taylor-series generator; the oracle's from
    # nested integer square roots.  Both must give the same numbers.
    path = os.path.join(ROOT, "paper_1512_02951_gb300", "csrc", "fds_cos_limbs.h")
    words = [int(x, 16) for x in re.findall(r"0x([0-9a-f]{8})u", open(path).read())]
    assert len(words) == 56
    for j in range(7):
        limbs = words[8 * j: 8 * j + 8]
        dev = sum(l << (32 * i) for i, l in enumerate(limbs))
        ora = exact.COS_FIXED[j + 1] >> (exact.FRAC_BITS - 256)
        assert abs(dev - ora) <= 2


def test_generated_header_is_up_to_date():
    import subprocess
    import sys

    csrc = os.path.join(ROOT, "paper_1512_02951_gb300", "csrc")
    out = subprocess.run([sys.executable, os.path.join(csrc, "gen_cos_limbs.py")],
                         capture_output=True, text=True, check=True).stdout
    assert out == open(os.path.join(csrc, "fds_cos_limbs.h")).read()


def test_plan_arguments_are_checked_on_the_host(lib):
    from paper_1512_02951_gb300 import _lib

    h = ctypes.c_void_p()
    assert lib.fds_plan_create(None, 0, ctypes.byref(h)) == -1
    d = (_lib.FdsImage * 1)()
    d[0].width, d[0].height, d[0].k, d[0].key_slot = 60, 64, 0, 0
    assert lib.fds_plan_create(d, 1, ctypes.byref(h)) == -1                 # width % 8
    d[0].width, d[0].key_slot = 64, 7
    assert lib.fds_plan_create(d, 1, ctypes.byref(h)) == -2                 # slot not registered
    d[0].key_slot, d[0].public_offset = 0, 8
    assert lib.fds_plan_create(d, 1, ctypes.byref(h)) in (-1, -2)           # misaligned offset
    assert lib.fds_plan_set_schedule(None, 1, 0, 0) == -1
    assert lib.fds_plan_set_direction_schedule(None, 0, 1, 0, 0) == -1
    assert lib.fds_plan_get_direction_schedule(None, 1, None, None, None) == -1
    assert lib.fds_plan_autotune_directions(None, None, None, None, None, 1, None) == -1
    n = ctypes.c_int64()
    assert lib.fds_plan_schedule_json(None, None, 0, ctypes.byref(n)) == -1
    assert lib.fds_plan_destroy(None) == 0


def test_full_encryption_arguments_are_checked_on_the_host(lib):
    key = bytes(16)
    assert lib.fds_encrypt_full(None, 16, 32, key, key, None) == -1          # null input
    assert lib.fds_encrypt_full(24, 32, 32, key, key, None) == -1            # not 16-aligned
    assert b"aligned" in lib.fds_last_error()
    assert lib.fds_encrypt_full(32, 48, 64, key, key, None) == -1            # partial overlap
    assert b"overlap" in lib.fds_last_error()
    assert lib.fds_encrypt_full(32, 32, 64, None, key, None) == -1           # null key


def test_packed_storage_sizes_and_checks(lib):
    from oracle import pack
    pub, priv, scr = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    for form in (11, 8):
        for (w, h, k) in [(64, 48, 0), (520, 40, 5), (8, 8, 63)]:
            assert lib.fds_sizes_packed(form, w, h, k, ctypes.byref(pub), ctypes.byref(priv), ctypes.byref(scr)) == 0
            assert (pub.value, priv.value) == pack.sizes(w, h, k, form)
            assert scr.value >= 2 * (w // 8) * (h // 8) * 3 * 64
    assert lib.fds_sizes_packed(10, 64, 64, 0, None, None, None) == -1
    key = bytes(16)
    assert lib.fds_protect_image_packed(11, 8, 64, 64, 0, key, key, 1, 24, 32, None) == -1   # private not 16-aligned
    assert lib.fds_protect_image_packed(11, 8, 64, 64, 0, key, key, 1, 32, None, None) == -1  # no scratch


def _primes(n):
    out, p = [], 2
    while len(out) < n:
        if all(p % q for q in out if q * q <= p):
            out.append(p)
        p += 1
    return out


def _icbrt(n):
    """floor(n^(1/3)) for a non-negative integer, by Newton's method on integers."""
    x = 1 << ((n.bit_length() + 2) // 3 + 1)
    while True:
        y = (2 * x + n // (x * x)) // 3
        if y >= x:
            break
        x = y
    while x ** 3 > n:
        x -= 1
    while (x + 1) ** 3 <= n:
        x += 1
    return x


def test_sha512_constants_follow_their_definition(lib):
    # FIPS 180-4: the first 64 bits of the fractional parts of the cube roots of the first 80
    # primes and of the square roots of the first 8
    import math

    from paper_1512_02951_gb300 import api

    kk, hh = api.sha512_constants()
    mask = (1 << 64) - 1
    ps = _primes(80)
    assert kk == [_icbrt(p << 192) & mask for p in ps]
    assert hh == [math.isqrt(p << 128) & mask for p in ps[:8]]


def test_strong_level_sizes_and_checks(lib):
    from paper_1512_02951_gb300 import api

    pub, priv, scr = api.sizes_strong(64, 48, 5)
    assert pub == 64 * 48 * 3 and priv == ofds.sizes(64, 48, 5)[1]
    assert scr >= priv + pub + ofds.sizes(64, 48, 5)[0] + priv
    u = ctypes.c_uint64()
    assert lib.fds_sizes_strong(60, 48, 5, ctypes.byref(u), ctypes.byref(u), ctypes.byref(u)) != 0
    key = bytes(16)
    # null / misaligned pointers fail on the host, before any device work
    assert lib.fds_protect_image_strong(None, 64, 48, 5, key, key, 16, 16, 16, None) != 0
    assert lib.fds_protect_image_strong(16, 64, 48, 5, key, key, 16, 24, 16, None) != 0
    assert lib.fds_restore_image_strong(16, 16, 64, 48, 64, key, key, 16, 16, None) != 0


def test_dwt_sizes_and_checks(lib):
    from paper_1512_02951_gb300 import api

    assert api.dwt_sizes(64, 48) == (5 * 48, 16 * 48, 60 * 48)
    u = ctypes.c_uint64()
    assert lib.fds_dwt_sizes(60, 48, ctypes.byref(u), ctypes.byref(u), ctypes.byref(u)) != 0
    key = bytes(16)
    assert lib.fds_dwt_protect(None, 64, 48, key, key, 16, 16, 16, None) != 0
    assert lib.fds_dwt_protect(16, 64, 48, key, key, 16, 24, 16, None) != 0     # misaligned level 2
    assert lib.fds_dwt_restore(16, 16, 16, 64, 44, key, key, 16, None) != 0      # H not a multiple of 8


def test_exact_round_diagnostic_rejects_vectors_outside_the_proven_range(lib):
    # the range check runs on the host before any device work
    bad = (ctypes.c_int32 * 8)(1 << 26, 0, 0, 0, 0, 0, 0, 0)
    out = (ctypes.c_int32 * 1)()
    assert lib.fds_debug_exact_round(bad, out, 1) == -1
    bad2 = (ctypes.c_int32 * 8)(0, 1 << 25, -(1 << 25), 0, 0, 0, 0, 0)
    assert lib.fds_debug_exact_round(bad2, out, 1) == -1
    assert lib.fds_debug_exact_round(None, None, -1) == -1


def test_failure_counter_maps_to_timeout_status(lib):
    # fds_sync reports bounded device waits that gave up: the mapping from a counter reading
    assert lib.fds_status_of_failures(0, 0) == 0
    assert lib.fds_status_of_failures(3, 3) == 0
    assert lib.fds_status_of_failures(5, 2) == 0
    assert lib.fds_status_of_failures(0, 1) == -5
    assert b"1 bounded device wait" in lib.fds_last_error()
    assert lib.fds_status_of_failures(7, 10) == -5
    assert lib.fds_last_error().startswith(b"3 ")
    assert lib.fds_debug_set_counters(None) == -1
