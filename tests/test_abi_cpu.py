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


def test_server_and_batch_argument_checks(lib):
    """The serving and batching constructors and the server calls check their
    arguments before any device call: out-of-range sizes and launch shapes,
    NULL handles and unknown streams return TRK_EINVAL with a reason."""
    out = C.c_void_p()
    good = dict(max_active=8, max_streams=8, max_pending=64, max_pixels=640 * 512, max_lambda=64, reserve=0,
                cluster=0, threads=0)

    def create(**kw):
        a = dict(good, **kw)
        return lib.server_create(a["max_active"], a["max_streams"], a["max_pending"], a["max_pixels"],
                                 a["max_lambda"], a["reserve"], a["cluster"], a["threads"], C.byref(out))

    for bad in (dict(max_active=0), dict(max_streams=0), dict(max_streams=4097), dict(max_pending=0),
                dict(max_pending=65537), dict(max_pixels=0), dict(max_pixels=1280 * 1280 + 1),
                dict(max_lambda=0), dict(reserve=-1), dict(cluster=9), dict(cluster=-1), dict(threads=48),
                dict(threads=288)):
        assert create(**bad) == TRK_EINVAL, bad
        assert out.value is None
        assert lib.tracker_last_error()
    assert lib.server_create(8, 8, 64, 640 * 512, 64, 0, 0, 0, None) == TRK_EINVAL
    sid = C.c_int32()
    assert lib.server_add_stream(None, None, 5, 0, C.byref(sid)) == TRK_EINVAL
    assert lib.server_remove_stream(None, 0) == TRK_EINVAL
    m = (C.c_uint8 * 16)()
    assert lib.server_submit(None, 0, m, None, 0, -1.0) == TRK_EINVAL
    a, q = C.c_int32(), C.c_int32()
    assert lib.server_step(None, C.byref(a), C.byref(q)) == TRK_EINVAL
    assert lib.server_poll(None, None, 0, 0, C.byref(a)) == TRK_EINVAL
    assert lib.server_destroy(None) == TRK_EINVAL
    assert lib.batch_create(None, None, None, 1, 0, 0, C.byref(out)) == TRK_EINVAL
    assert out.value is None
    lam = (C.c_int32 * 1)(64)
    trackers = (C.c_void_p * 1)()
    assert lib.batch_create(trackers, None, lam, 0, 0, 0, C.byref(out)) == TRK_EINVAL
    assert lib.batch_create(trackers, None, None, 1, 0, 0, C.byref(out)) == TRK_EINVAL
    assert lib.batch_create(trackers, None, lam, 1, 0, 0, None) == TRK_EINVAL
