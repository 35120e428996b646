"""Failure handling on the GPU without a GPU fault: a bounded device wait
that runs out.

The overlapped final merge of larger-side rounds (Fig. 3 "out" with its
half-size buffer) is the one place where blocks wait on one another.  The
test hook QMS_FLAG_TEST_WITHHOLD makes its first tile never publish its
completion flag; with qms_options.spin_limit = 1 every wait on that tile
gives up after two polls, the error bit stops all later waits, and the sort
returns QMS_ETIMEOUT.  The context stays usable: the next ordinary sort must
still equal the plain definition of the result."""
import numpy as np
import pytest

import oracle
import qms_inputs as gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1804_10062_gb300 as q
    q.lib()
    return q


def _dev(a):
    return torch.from_numpy(a.view(np.int32).copy()).cuda()


@pytest.mark.parametrize("host_driven", [True, False])
def test_withheld_flag_times_out_and_next_sort_is_clean(q, host_driven):
    n = (1 << 20) + 3
    k = gen.keys("uniform", "u32", n, 71)
    d = _dev(k)
    with pytest.raises(q.QmsError) as ei:
        q.qms_sort(d, side="larger", host_driven=host_driven, spin_limit=1, test_withhold=True,
                   dtype="u32")
    assert ei.value.code == q.QMS_ETIMEOUT
    torch.cuda.synchronize()
    for side in ("larger", "fig3"):
        k2 = gen.keys("uniform", "u32", n, 72)
        d2 = _dev(k2)
        q.qms_sort(d2, side=side, host_driven=host_driven, dtype="u32")
        out = d2.cpu().numpy().view(np.uint32)
        assert out.tobytes() == oracle.reference_sorted(k2).tobytes(), side


def test_spin_limit_alone_does_not_time_out(q):
    # A small limit with every flag published: waits may still give up if a
    # tile is slow, so only the default limit is checked for success here,
    # and a limit of 1 either succeeds or reports QMS_ETIMEOUT (never a
    # wrong result reported as success).
    n = (1 << 20) + 3
    k = gen.keys("uniform", "u32", n, 73)
    d = _dev(k)
    q.qms_sort(d, side="larger", dtype="u32")
    assert d.cpu().numpy().view(np.uint32).tobytes() == oracle.reference_sorted(k).tobytes()
    d = _dev(k)
    try:
        q.qms_sort(d, side="larger", spin_limit=1, dtype="u32")
    except q.QmsError as e:
        assert e.code == q.QMS_ETIMEOUT
    else:
        assert d.cpu().numpy().view(np.uint32).tobytes() == oracle.reference_sorted(k).tobytes()
