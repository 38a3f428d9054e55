"""Pins of the oracle's exact rounding (Sect. 6.4.3 reading: round half away from zero of the
exact value) against closed forms, algebraic identities and 50-digit brute force."""
import math

import numpy as np
import pytest

from oracle import dct, exact, fds


def _mp():
    return pytest.importorskip("mpmath")


def _hp_dct(block, mp):
    """F[u, v] at 50 digits, straight from the defining double sum."""
    mp.mp.dps = 50
    out = [[None] * 8 for _ in range(8)]
    for u in range(8):
        cu = mp.sqrt(mp.mpf(1) / 2) if u == 0 else mp.mpf(1)
        for v in range(8):
            cv = mp.sqrt(mp.mpf(1) / 2) if v == 0 else mp.mpf(1)
            s = mp.mpf(0)
            for y in range(8):
                for x in range(8):
                    s += int(block[y][x]) * mp.cos((2 * y + 1) * u * mp.pi / 16) \
                        * mp.cos((2 * x + 1) * v * mp.pi / 16)
            out[u][v] = cu * cv * s / 4
    return out


def _hp_idct(coefs, mp):
    mp.mp.dps = 50
    out = [[None] * 8 for _ in range(8)]
    for y in range(8):
        for x in range(8):
            s = mp.mpf(0)
            for u in range(8):
                cu = mp.sqrt(mp.mpf(1) / 2) if u == 0 else mp.mpf(1)
                for v in range(8):
                    cv = mp.sqrt(mp.mpf(1) / 2) if v == 0 else mp.mpf(1)
                    s += cu * cv * int(coefs[u][v]) * mp.cos((2 * y + 1) * u * mp.pi / 16) \
                        * mp.cos((2 * x + 1) * v * mp.pi / 16)
            out[y][x] = s / 4
    return out


def _hp_round(val, mp):
    """round half away from zero of a 50-digit value that is not within 1e-30 of a tie."""
    a = abs(val)
    fl = mp.floor(a)
    assert abs(a - fl - mp.mpf(1) / 2) > mp.mpf(10) ** -30
    r = int(fl) + (1 if a - fl > mp.mpf(1) / 2 else 0)
    return r if val >= 0 else -r


def test_fold_cos():
    for m in range(-70, 71):
        j, s = exact.fold_cos(m)
        assert 0 <= j <= 8
        assert abs(s * math.cos(j * math.pi / 16) - math.cos(m * math.pi / 16)) < 1e-13


def test_fixed_cosines_against_float_and_identities():
    c = exact.COS_FIXED
    one = 1 << exact.FRAC_BITS
    for j in range(9):
        assert abs(c[j] / one - math.cos(j * math.pi / 16)) < 1e-15
    # double-angle and complement identities, exact to a few units of 2^-FRAC_BITS
    for j in range(1, 5):
        lhs = 2 * c[j] * c[j] - one * one          # (2 c(j)^2 - 1) at scale 2^(2 FRAC_BITS)
        assert abs(lhs - c[2 * j] * one) < 8 * one
    for j in range(1, 8):
        assert abs(c[j] * c[j] + c[8 - j] * c[8 - j] - one * one) < 8 * one


def test_basis_coordinates_represent_the_basis_products():
    b = dct.basis_matrix()
    cj = np.array([math.cos(j * math.pi / 16) for j in range(8)])
    val = exact.K @ cj                                         # [u, v, y, x]
    want = 8 * np.einsum("uy,vx->uvyx", b, b)
    assert np.abs(val - want).max() < 1e-14
    # every product has exactly two +-1 terms (one may vanish through c(8) = 0)
    assert np.abs(exact.K).sum(axis=-1).max() <= 2


def test_forward_coordinates_agree_with_float():
    rng = np.random.default_rng(11)
    cj = np.array([math.cos(j * math.pi / 16) for j in range(8)])
    for _ in range(20):
        p = rng.integers(0, 256, (8, 8))
        f = dct.dct2(p)
        for u in range(8):
            for v in range(8):
                n = exact.forward_coords(p, u, v)
                assert abs((n @ cj) / 8 - f[u, v]) < 1e-9


def test_rational_positions_and_dc_closed_form():
    rng = np.random.default_rng(12)
    blocks = rng.integers(0, 256, (400, 8, 8))
    q, _ = fds.quantised_dct(blocks)
    for i, p in enumerate(blocks):
        s = int(p.sum())
        n = exact.forward_coords(p, 0, 0)
        assert n[0] == s and not n[1:].any()                  # 8 F[0,0] = S
        assert q[i, 0, 0] == (s + 4) // 8                      # half away from zero, S >= 0
        for u, v in ((0, 4), (4, 0), (4, 4)):
            assert not exact.forward_coords(p, u, v)[1:].any()  # always rational


@pytest.mark.parametrize("s_mod", range(8))
def test_dc_tie_iff_sum_is_4_mod_8(s_mod):
    p = np.zeros((8, 8), dtype=np.int64)
    p[0, 0] = 8 * 5 + s_mod                                    # S = 40 + s_mod
    n = exact.forward_coords(p, 0, 0)
    tie = (not n[1:].any()) and n[0] % 8 == 4
    assert tie == (s_mod == 4)
    q, _ = fds.quantised_dct(p)
    assert q[0, 0] == (40 + s_mod + 4) // 8


def test_negative_rational_tie_rounds_away_from_zero():
    # 8 F[0,4] = sum_y sum_x p w(x), w = (1,-1,-1,1,1,-1,-1,1): choose it = -12 -> F = -1.5
    p = np.zeros((8, 8), dtype=np.int64)
    p[0, 1] = 12
    n = exact.forward_coords(p, 0, 4)
    assert n[0] == -12 and not n[1:].any()
    q, f = fds.quantised_dct(p)
    assert abs(f[0, 4] + 1.5) < 1e-12
    assert q[0, 4] == -2
    p[0, 1] = 20                                               # F[0,4] = -2.5 -> -3
    assert fds.quantised_dct(p)[0][0, 4] == -3
    p[0, 1] = 0
    p[0, 0] = 12                                               # F[0,4] = +1.5 -> 2
    assert fds.quantised_dct(p)[0][0, 4] == 2


def test_irrational_position_ties_exist_and_round_away():
    # ties at (2,2) live in Q(sqrt 2): search seeded small blocks for N_j = 0 (j > 0), N_0 = 4 mod 8
    rng = np.random.default_rng(13)
    blocks = rng.integers(0, 3, (200000, 8, 8))
    n = np.einsum("myx,yxj->mj", blocks, exact.K[2, 2])
    hit = np.nonzero((n[:, 1:] == 0).all(axis=1) & (n[:, 0] % 8 == 4))[0]
    assert hit.size > 0
    for i in hit[:20]:
        q, f = fds.quantised_dct(blocks[i])
        val = n[i, 0] / 8
        assert abs(f[2, 2] - val) < 1e-12
        assert q[2, 2] == int(math.copysign(math.floor(abs(val) + 0.5), val))


def test_exact_sign_against_high_precision():
    mp = _mp()
    mp.mp.dps = 80
    rng = np.random.default_rng(14)
    cs = [mp.cos(j * mp.pi / 16) for j in range(8)]
    for _ in range(300):
        n = rng.integers(-40000, 40000, 7)
        val = sum(int(n[j]) * cs[j + 1] for j in range(7))
        a0 = -int(mp.nint(val)) + int(rng.integers(-1, 2))      # make the total small
        tot = a0 + val
        if abs(tot) < mp.mpf(10) ** -60:
            continue
        assert exact.exact_sign(a0, n) == (1 if tot > 0 else -1)
    assert exact.exact_sign(-3, [0] * 7) == -1
    assert exact.exact_sign(0, [0] * 7) == 0


def test_near_relations_fixture_is_tiny_nonzero_and_signed_right():
    # tests/golden/exact_near_relations.txt: N_0 + sum_j N_j cos(j pi/16) nonzero, tiny, its
    # sign the oracle's, and -- shifted onto a half-integer boundary -- closer to it than a
    # 64-bit fixed-point evaluation can resolve (what makes the device escalate)
    from conftest import read_golden
    mp = _mp()
    mp.mp.dps = 60
    cs = [mp.cos(j * mp.pi / 16) for j in range(8)]
    rows = [[int(t) for t in ln.split("#")[0].split()] for ln in read_golden("exact_near_relations.txt")]
    assert len(rows) >= 24
    for n in rows:
        val = n[0] + sum(n[j] * cs[j] for j in range(1, 8))
        assert mp.mpf(2) ** -100 < abs(val) < mp.mpf(2) ** -55
        assert exact.exact_sign(n[0], n[1:]) == (1 if val > 0 else -1)
        assert sum(abs(t) for t in n[1:]) * mp.mpf(2) ** -62 > abs(val)   # below the 64-bit error bound
        assert max(abs(t) for t in n) <= 32640                            # forward-transform range


def test_forward_rounding_against_brute_force():
    mp = _mp()
    rng = np.random.default_rng(15)
    # seeded blocks with some coefficient inside the 1e-6 band of a half-integer, plus plain ones
    cand = rng.integers(0, 256, (400000, 8, 8))
    f = dct.dct2(cand)
    d = np.abs(f - np.floor(f) - 0.5)
    # non-tie values inside the float64 band: decided by exact_sign
    near = np.nonzero(((d > 1e-11) & (d < fds.BAND)).any(axis=(1, 2)))[0][:4]
    assert near.size >= 2
    picks = list(cand[near]) + list(rng.integers(0, 256, (2, 8, 8)))
    for p in picks:
        q, _ = fds.quantised_dct(p)
        hp = _hp_dct(p, mp)
        for u in range(8):
            for v in range(8):
                n = exact.forward_coords(p, u, v)
                if not n[1:].any() and n[0] % 8 == 4:
                    continue                                    # exact ties: closed-form tests
                assert q[u, v] == _hp_round(hp[u][v], mp), (u, v)


def test_inverse_rounding_against_brute_force():
    mp = _mp()
    rng = np.random.default_rng(16)
    cand = rng.integers(-60, 60, (400000, 8, 8))
    cand[:, 0, 0] = rng.integers(0, 2041, 400000)
    p = dct.idct2(cand)
    d = np.abs(p - np.floor(p) - 0.5)
    near = np.nonzero(((d > 1e-11) & (d < fds.BAND)).any(axis=(1, 2)))[0][:3]
    assert near.size >= 2
    picks = list(cand[near]) + list(cand[:1])
    for c in picks:
        r = fds.quantised_idct(c)
        hp = _hp_idct(c, mp)
        for y in range(8):
            for x in range(8):
                m = exact.inverse_coords(c, y, x)
                if not m[1:].any() and m[0] % 8 == 4:
                    continue
                assert r[y, x] == _hp_round(hp[y][x], mp), (y, x)


def test_inverse_pixel_ties_round_away_from_zero():
    # a DC-only coefficient block q gives 8 p = q at every pixel: q = 4 mod 8 is a tie
    for qdc, want in ((20, 3), (-20, -3), (12, 2), (2044, 256)):
        c = np.zeros((8, 8), dtype=np.int64)
        c[0, 0] = qdc
        m = exact.inverse_coords(c, 3, 5)
        assert m[0] == qdc and not m[1:].any()
        assert (fds.quantised_idct(c) == want).all()


@pytest.mark.parametrize("inverse", [False, True])
def test_exact_path_agrees_with_float_where_float_is_unambiguous(inverse, monkeypatch):
    # widen the band so that the exact path decides almost every entry; away from ties the
    # float64 decision is certainly right, so both must agree
    rng = np.random.default_rng(17)
    if inverse:
        x = rng.integers(-200, 200, (40, 8, 8))
        narrow = fds.quantised_idct(x)
        monkeypatch.setattr(fds, "BAND", 0.45)
        wide = fds.quantised_idct(x)
    else:
        x = rng.integers(0, 256, (40, 8, 8))
        narrow = fds.quantised_dct(x)[0]
        monkeypatch.setattr(fds, "BAND", 0.45)
        wide = fds.quantised_dct(x)[0]
    assert np.array_equal(narrow, wide)
