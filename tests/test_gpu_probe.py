"""The integer-issue probe (the fitness kernel's roofline denominator): the
measured rate is close to the figure derived from the SM count, 64 INT32
lanes per SM per clock and the device's maximum SM clock."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_11404_gb300 import build
    build.build()
    from paper_2603_11404_gb300 import api as a
    return a


def test_probe_measures_the_integer_issue_peak(api):
    r = api.probe_int_issue(2000)
    assert r["ms"] > 0.5
    # the SMs may run below their maximum clock (power cap), never much above it
    assert 0.5 * r["derived_tops"] < r["tops"] < 1.05 * r["derived_tops"], r


def test_probe_rejects_bad_arguments(api):
    from paper_2603_11404_gb300._abi import TrkError
    with pytest.raises(TrkError):
        api.probe_int_issue(0)
