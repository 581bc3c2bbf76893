"""The allocation-free dose entry point (dd_per_probe_dose_noalloc).

Callers that cannot allocate device memory while they run -- for instance an
acquisition loop that reserves its GPU memory budget before the scan begins -- use this
entry point; it keeps its scratch in the library's fixed 8 MiB device array.  The tests
call it through the C-ABI twice in a row (a larger scan, then a smaller one, so stale
scratch from the first call would show up in the second) and compare each result with
dd_per_probe_dose at the tolerances the other GPU tests use; the largest accepted scan
(128 x 128 = 16384 visits, whose FP64 scratch takes about 8.0 of the 8.4 MB) is also
compared with the oracle on seeded targets.  This file is collected last so that a stop
at the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2507_00294_gb300 import binding as b
from paper_2507_00294_gb300 import workloads as w
from parity_util import assert_fp64, assert_mixed, oracle_dose

pytestmark = pytest.mark.gpu

FP64_RTOL = 1e-12
MIXED_RTOL = 1e-5


@pytest.mark.parametrize("prec,rtol", [("fp64", FP64_RTOL), ("mixed", MIXED_RTOL)])
def test_noalloc_dose_matches_dose_twice(cuda, prec, rtol):
    import torch
    specs = [w.ScanSpec(128, 128), w.ScanSpec(64, 64),
             w.ScanSpec(23, 19, order=w.RANDOM, seed=8, keep_fraction=0.7)]
    for spec in specs:
        scan = b.Scan(spec)
        n = len(scan)
        ref = b.dd_per_probe_dose(scan, prec, device=cuda)
        out = torch.full((n,), float("nan"), dtype=torch.float64, device=cuda)
        b.dd_per_probe_dose_noalloc(scan, out, prec)
        torch.cuda.synchronize()
        got, exp = out.cpu().numpy(), ref.cpu().numpy()
        assert got[0] == 0.0 and np.all(np.isfinite(got))
        np.testing.assert_allclose(got[1:], exp[1:], rtol=rtol, atol=0)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_dose_at_the_limit_against_the_oracle(cuda, prec):
    """16384 visits, the most the fixed scratch accepts: seeded targets (and the first and
    last visits) against the oracle."""
    import torch
    spec = w.ScanSpec(128, 128, order=w.SERPENTINE)
    scan = b.Scan(spec)
    n = len(scan)
    assert n == 16384
    out = torch.full((n,), float("nan"), dtype=torch.float64, device=cuda)
    b.dd_per_probe_dose_noalloc(scan, out, prec)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    rng = np.random.default_rng(41)
    targets = np.unique(np.concatenate([[1, 2, 127, 128, 129, n - 1],
                                        rng.choice(np.arange(1, n), 1024, replace=False)]))
    ref = oracle_dose(spec, targets)
    assert got[0] == 0.0
    if prec == "fp64":
        assert_fp64(got[targets], ref, "noalloc dose 128x128 fp64")
    else:
        assert_mixed(got[targets], ref, ref.max(), "noalloc dose 128x128 mixed")


def test_noalloc_dose_rejects_oversize_and_host_output(cuda):
    import torch
    big = b.Scan(w.ScanSpec(129, 128))             # 16512 visits > 16384
    out = torch.empty(len(big), dtype=torch.float64, device=cuda)
    with pytest.raises(b.DDError) as e:
        b.dd_per_probe_dose_noalloc(big, out, "mixed")
    assert e.value.status == b.DD_EINVAL and "16384" in str(e.value)
    small = b.Scan(w.ScanSpec(4, 4))
    with pytest.raises(b.DDError) as e:
        b.dd_per_probe_dose_noalloc(small, np.empty(16), "mixed")
    assert e.value.status == b.DD_EINVAL
