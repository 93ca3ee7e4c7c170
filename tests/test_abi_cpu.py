"""The C-ABI library on a machine without a GPU: it builds, loads, exports every
function include/tracker.h declares with the argument list the binding uses,
and rejects bad arguments on the host (TRK_EINVAL, nothing enqueued) before
any device work.  No kernel is launched here."""
import ctypes as C

import pytest

from paper_2603_11404_gb300 import _abi, build

TRK_OK, TRK_EINVAL = 0, 1


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _abi.lib()


def test_every_declared_function_is_exported_and_bound(lib):
    declared = _abi.declared_symbols()
    assert len(declared) > 40
    raw = C.CDLL(_abi.LIB)
    missing = [n for n in declared if not hasattr(raw, n)]
    assert not missing, missing
    # every declared status-returning function has the binding's argument list
    special = {"trk_status_string", "tracker_last_error", "server_now"}
    unbound = [n for n in declared if n not in _abi.SIGNATURES and n not in special]
    assert not unbound, unbound
    # and the binding names nothing the header does not declare
    assert not [n for n in _abi.SIGNATURES if n not in declared]


def test_status_strings(lib):
    assert lib.trk_status_string(TRK_OK) == b"ok"
    assert lib.trk_status_string(TRK_EINVAL) == b"invalid argument"
    assert lib.trk_status_string(99) == b"unknown status"


def test_host_side_argument_checks(lib):
    """Calls that fail their argument checks return TRK_EINVAL with a reason and
    touch no device state, so they run without a GPU."""
    out = C.c_void_p()
    assert lib.tracker_create(None, 0, None, None, None, C.byref(out)) == TRK_EINVAL
    assert out.value is None
    assert lib.tracker_last_error()
    assert lib.eval_population(None, None, 4, None, None, None, None) == TRK_EINVAL
    assert lib.cmaes_step(None, None, None) == TRK_EINVAL
    n = C.c_size_t(0)
    assert lib.cmaes_save(None, None, C.byref(n), None) == TRK_EINVAL
    tops = C.c_double()
    assert lib.trk_probe_int_issue(0, C.byref(tops), None, None) == TRK_EINVAL
    assert b"iters" in lib.tracker_last_error()
    assert lib.trk_probe_int_issue(100, None, None, None) == TRK_EINVAL


def test_image_above_the_bitmap_limit_is_rejected(lib):
    """One row more than TRK_MAX_PIXELS (1280 x 1280: the bitmap must fit one
    CTA's shared memory) is refused by tracker_create before any allocation."""
    from paper_2603_11404_gb300 import api, workload as wl
    K = wl.Intrinsics(1600.0, 1600.0, 640.0, 640.5, 1280, 1281)
    with pytest.raises(_abi.TrkError) as e:
        api.Tracker(wl.make_scene("c1", "c1", K=K), lambda_max=4)
    assert e.value.status == TRK_EINVAL
