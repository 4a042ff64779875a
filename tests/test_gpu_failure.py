"""Failure detection on the GPU without a GPU fault: the bounded waits of
the pipelined kernels.  Every wait for a staged copy gives up after a time
limit, records a bit in the handle's device error word and lets its block
return; the host then reports FFTLB_ERR_TIMEOUT.  fftlb_debug_wait_test
makes that happen on purpose: each stage first runs a kernel whose blocks
wait, through the same bounded-wait code and with a 1 ms limit, on a
shared-memory barrier that nothing completes (no copy is issued there, so
nothing is in flight when the blocks return).  The context stays usable."""
import numpy as np
import pytest

from gpu_common import lib, slab64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fl():
    return lib()


def test_wait_that_nothing_completes_reports_timeout(fl):
    fields, kw = slab64()
    p = fl.params(precision=32, check_every=1, **kw)
    h = fl.Handle(p)
    try:
        h.set_fields(*fields)
        assert h.step(2) == 2                       # normal steps
        h.debug_wait_test(1_000_000)                # 1 ms limit
        with pytest.raises(fl.FFTLBError) as ei:
            h.step(1)
        assert ei.value.status == fl.ERR_TIMEOUT
        assert "wait" in str(ei.value)
        # the word stays set: later reads report the timeout too
        with pytest.raises(fl.FFTLBError) as ei2:
            h.invariants()
        assert ei2.value.status == fl.ERR_TIMEOUT
    finally:
        h.close()                                   # destroys cleanly
    # the context is still usable: a new handle steps and matches a clean run
    with fl.Handle(p) as h2:
        h2.set_fields(*fields)
        h2.step(3)
        inv = h2.invariants()
    assert np.isfinite(inv["mass"]) and inv["time"] == pytest.approx(3e-5)


def test_wait_test_rejects_bad_limits(fl):
    fields, kw = slab64()
    with fl.Handle(fl.params(precision=32, **kw)) as h:
        for ns in (-1, 10, 10 ** 10):
            with pytest.raises(fl.FFTLBError) as ei:
                h.debug_wait_test(ns)
            assert ei.value.status == fl.ERR_ARG
        h.debug_wait_test(0)                        # off
        h.set_fields(*fields)
        h.step(1)
