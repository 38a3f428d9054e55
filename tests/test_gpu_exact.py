"""The device's exact rounding step (round half away from zero of the exact value, the reading
of Sect. 6.4.3) on coordinate vectors, through the C ABI, against oracle/exact.py.

The fused kernels reach this step only for values within their float32 guard of a
half-integer, and on natural images its 64-bit first evaluation always decides.  Here it gets
vectors that the 64-bit evaluation cannot decide: integer relations of 1, cos(pi/16), ..,
cos(7 pi/16) with a tiny nonzero value (found by lattice reduction, tests/golden/), shifted
onto rounding boundaries of both signs.  Every one of them must go through the 256-bit
evaluation (counter 1 of fds_counters) and come out equal to the oracle's decision."""
import numpy as np
import pytest

from conftest import read_golden
from oracle import exact, fds as ofds

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_02951_gb300 import api as _api, build

    build.build()
    _api.init(0)
    return _api


def relations():
    return [[int(t) for t in ln.split("#")[0].split()] for ln in read_golden("exact_near_relations.txt")]


def _oracle_round(coords):
    """The oracle's decision; its float64 hint is the exact value rounded once."""
    v = coords[0] * (1 << exact.FRAC_BITS) + sum(coords[j] * exact.COS_FIXED[j] for j in range(1, 8))
    approx = v / float(1 << (exact.FRAC_BITS + 3))
    return exact.round_half_away(approx, coords, ofds.BAND)


def _shifted(n, m):
    return [n[0] + 4 + 8 * m] + list(n[1:])


def test_relations_force_the_wide_evaluation(api):
    rel = relations()
    assert len(rel) >= 24
    vecs, ms = [], []
    for n in rel:
        for sgn in (1, -1):
            for m in (0, 1, -1, -3, 7, 254, -255):
                vecs.append(_shifted([sgn * t for t in n], m))
                ms.append(m)
    api.counters(reset=True)
    got = api.debug_exact_round(vecs)
    red, esc, fail = api.counters()
    want = [_oracle_round(v) for v in vecs]
    bad = [(v, g, w) for v, g, w in zip(vecs, got, want) if g != w]
    assert not bad, bad[:5]
    assert fail == 0
    assert esc == len(vecs), (esc, len(vecs))          # every one needed the 256-bit step
    # m = 0: V = 1/2 + s/8 rounds to 1 or 0 by the sign of s; both occur (relations of both signs)
    assert {g for m, g in zip(ms, got) if m == 0} == {0, 1}


def test_exact_ties_and_plain_values(api):
    rng = np.random.default_rng(21)
    vecs = []
    for m in range(-40, 40):                            # exact ties: away from zero, no escalation
        vecs.append([8 * m + 4] + [0] * 7)
    for _ in range(3000):                               # forward-transform magnitudes
        n = [int(t) for t in rng.integers(-32640, 32641, 8)]
        vecs.append(n)
    for _ in range(3000):                               # near boundaries, decided in 64 bits
        n = [0] + [int(t) for t in rng.integers(-3000, 3001, 7)]
        s = sum(n[j] * exact.COS_FIXED[j] for j in range(1, 8)) >> exact.FRAC_BITS
        n[0] = int(4 - s + 8 * rng.integers(-200, 200))
        vecs.append(n)
    api.counters(reset=True)
    got = api.debug_exact_round(vecs)
    want = [_oracle_round(v) for v in vecs]
    assert got == want
    red, esc, fail = api.counters()
    assert fail == 0 and esc == 0
    assert got[:80] == [m + 1 if m >= 0 else m for m in range(-40, 40)]


def test_out_of_range_vectors_are_rejected(api):
    from paper_1512_02951_gb300 import _lib
    with pytest.raises(_lib.FdsError):
        api.debug_exact_round([[1 << 26] + [0] * 7])
    with pytest.raises(_lib.FdsError):
        api.debug_exact_round([[0, 1 << 25, 1 << 25, 0, 0, 0, 0, 0]])
