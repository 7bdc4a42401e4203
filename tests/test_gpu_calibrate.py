"""Measurement kernels on the GPU: every configuration runs, its IR's counts are the
ones the CUDA kernel performs (checked on closed forms here), and a quick fit of the
model to this GPU predicts the measurement set itself within a loose bound."""
import numpy as np
import pytest

from paper_1604_04997_gb300 import binding as B
from paper_1604_04997_gb300 import calibrate as C
from paper_1604_04997_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    c = B.Context(0)
    yield c
    c.close()


def test_every_probe_kind_times(ctx):
    cases = C.measurement_set(quick=True)[::3] + C.test_set(quick=True)[::2]
    t = C.time_cases(cases, runs=5, skip=1)
    assert (t > 0).all() and np.isfinite(t).all()


def test_probe_counts_closed_forms(ctx):
    n = 1 << 20
    cases = [C.Case(W.Probe("copy"), (n,), ""), C.Case(W.Probe("sum4", gx=512), (n,), ""),
             C.Case(W.Probe("vsa", 3), (n,), ""), C.Case(W.Probe("filled", 2, 256), (n,), ""),
             C.Case(W.Probe("arith", 1, 512, 32, 16), (1024,), ""),
             C.Case(W.Probe("matmul", gx=32, gy=32), (256, 128, 64), ""),
             C.Case(W.Probe("empty", gx=16, gy=16), (1000,), "")]
    F = C.features(ctx, cases)
    assert (F[0, 17], F[0, 24]) == (n, n)                       # one stride-1 load and store each
    assert (F[1, 17], F[1, 3], F[1, 1]) == (4 * n, 3 * n, n // 512)
    assert (F[2, 19], F[2, 26], F[2, 4], F[2, 3]) == (2 * n, n, 2 * n, n)
    assert (F[3, 18], F[3, 3]) == (2 * 256 * n, 2 * 256 * n)    # filled stride-2 loads
    assert F[4, 4] == 1024 * 1024 * 512 * 8
    assert (F[5, 3], F[5, 4], F[5, 2]) == (256 * 128 * 64, 256 * 128 * 64, 2 * (64 // 32) * (256 // 32) * (128 // 32))
    assert (F[6, 1], F[6].sum() - F[6, 0] - F[6, 1]) == (63 * 63, 0)


def test_quick_calibration(ctx):
    r = C.calibrate(ctx, quick=True, runs=8, skip=2)
    assert r["fit_status"] in (0, 1)
    assert r["measurement"]["geomean_rel_err"] < 0.5
    assert np.isfinite(r["test"]["geomean_rel_err"])
    sel = r["selection"]
    for rows in sel["families"].values():
        for row in rows:
            assert sorted(row["predicted_order"]) == list(range(len(row["candidates"])))
            assert row["top1_slowdown"] >= 0 and row["top2_slowdown"] <= row["top1_slowdown"]
            assert row["predicted_s"] == sorted(row["predicted_s"])


def test_integer_issue_rate_probe():
    """The integer issue-rate probe: positive, below the derived bound of 128 lane
    operations per SM per clock at the maximum clock, and repeatable."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    props = torch.cuda.get_device_properties(0)
    bound = props.multi_processor_count * 128 * 2.2e9
    a, b = B.pmm_int_issue_rate(), B.pmm_int_issue_rate()
    assert 0.05 * bound < a <= bound and abs(a - b) <= 0.1 * a
