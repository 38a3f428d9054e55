"""A bounded device wait that gave up surfaces as FDS_E_TIMEOUT from fds_sync.

No wait is made to give up: the counter the kernels add to is written by a test hook, and
fds_sync must report the increase once, then return to FDS_OK."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_sync_reports_a_failure_count_once():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_02951_gb300 import _lib, api, build

    build.build()
    api.init(0)
    api.counters(reset=True)
    api.sync()                                       # nothing failed
    api.debug_set_counters([0, 0, 2])
    with pytest.raises(_lib.FdsError) as err:
        api.sync()
    assert err.value.code == _lib.FDS_E_TIMEOUT
    assert "2 bounded device wait" in str(err.value)
    api.sync()                                       # reported once
    api.debug_set_counters([0, 0, 3])
    with pytest.raises(_lib.FdsError):
        api.sync()
    api.counters(reset=True)                         # leave the counters clean for the other tests
    api.sync()
    assert api.counters() == (0, 0, 0)
