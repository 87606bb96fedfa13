"""Failure detection, host side: the bounded-wait rule that every spin wait
of the CUDA kernels follows (csrc/wait.h), compiled for the host and driven
by CPU threads.  A barrier that gets one arrival fewer than it expects must
make the waits give up within their limit and raise the shared abort flag;
the other waits of the same CTA must then give up at once instead of
running out their own limits; a drain wait on a flag of its own must still
see work that completes after the abort."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1201_6062_gb300", "csrc")
MS = 1_000_000


@pytest.fixture(scope="module")
def waitlib(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("wait") / "libwait.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread", "-I", CSRC, "-o", out,
                           os.path.join(ROOT, "tests", "helpers", "wait_capi.cpp")])
    lib = ctypes.CDLL(out)
    lib.wait_scenario.restype = ctypes.c_int
    return lib


def run(lib, expected, given, delay_ns, timeouts, own=None, abort_after=-1):
    W = len(timeouts)
    to = np.asarray(timeouts, np.int64)
    own = np.asarray(own if own is not None else [0] * W, np.int32)
    ok = np.zeros(W, np.int32)
    el = np.zeros(W, np.int64)
    ab = ctypes.c_int(0)
    P = ctypes.POINTER
    lib.wait_scenario(W, expected, given, ctypes.c_long(delay_ns), to.ctypes.data_as(P(ctypes.c_long)),
                      own.ctypes.data_as(P(ctypes.c_int)), ctypes.c_long(abort_after),
                      ok.ctypes.data_as(P(ctypes.c_int)), el.ctypes.data_as(P(ctypes.c_long)), ctypes.byref(ab))
    return ok, el, ab.value


def test_all_arrivals_complete_the_phase(waitlib):
    ok, el, ab = run(waitlib, 3, 3, 2 * MS, [2000 * MS] * 4)
    assert ok.tolist() == [1] * 4 and ab == 0


def test_a_missing_arrival_times_out_and_raises_the_abort_flag(waitlib):
    ok, el, ab = run(waitlib, 3, 2, 1 * MS, [30 * MS] * 4)
    assert ok.tolist() == [0] * 4 and ab == 1
    assert el.min() >= 30 * MS                     # nobody gave up before the limit
    assert el.max() < 1000 * MS                    # and every wait ended


def test_the_other_waits_of_the_cta_follow_the_abort_flag(waitlib):
    # waiter 0 has a short limit; the others would wait 20 s on their own
    ok, el, ab = run(waitlib, 2, 0, 0, [20 * MS] + [20000 * MS] * 5)
    assert ok.tolist() == [0] * 6 and ab == 1
    assert el.max() < 2000 * MS


def test_an_abort_from_elsewhere_ends_every_wait(waitlib):
    ok, el, ab = run(waitlib, 1, 0, 0, [20000 * MS] * 3, abort_after=20 * MS)
    assert ok.tolist() == [0] * 3 and ab == 1
    assert el.min() >= 20 * MS and el.max() < 2000 * MS


def test_a_drain_wait_on_its_own_flag_sees_late_completion(waitlib):
    # waiter 0 times out and aborts; waiter 1 (its own flag) keeps waiting for
    # the arrivals that still come, as the kernels' drains of copies in flight do
    ok, el, ab = run(waitlib, 2, 2, 60 * MS, [20 * MS, 5000 * MS], own=[0, 1])
    assert ok.tolist() == [0, 1] and ab == 1
    assert el[1] >= 120 * MS
