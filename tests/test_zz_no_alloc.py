"""The allocation-free dose entry point (dd_per_probe_dose_noalloc).

Callers that cannot allocate device memory while they run -- for instance an
acquisition loop that reserves its GPU memory budget before the scan begins -- use this
entry point; it keeps its scratch in the library's fixed 8 MiB device array.  The test
calls it through the C-ABI twice in a row (a larger scan, then a smaller one, so stale
scratch from the first call would show up in the second) and compares each result with
dd_per_probe_dose at the tolerances the other GPU tests use.  This file is collected
last so that a stop at the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2507_00294_gb300 import binding as b
from paper_2507_00294_gb300 import workloads as w

pytestmark = pytest.mark.gpu

FP64_RTOL = 1e-12
MIXED_RTOL = 1e-5


@pytest.mark.parametrize("prec,rtol", [("fp64", FP64_RTOL), ("mixed", MIXED_RTOL)])
def test_noalloc_dose_matches_dose_twice(cuda, prec, rtol):
    import torch
    specs = [w.ScanSpec(64, 64), w.ScanSpec(23, 19, order=w.RANDOM, seed=8, keep_fraction=0.7)]
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
