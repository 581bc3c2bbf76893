"""GPU dwell-start dose (dd_per_probe_dose) against the CPU oracle, through the C-ABI."""
import numpy as np
import pytest

from paper_2507_00294_gb300 import binding as b
from paper_2507_00294_gb300 import workloads as w
from parity_util import assert_fp64, assert_mixed, oracle_dose

pytestmark = pytest.mark.gpu


def gpu_dose(spec, prec):
    import torch
    scan = b.Scan(spec)
    out = b.dd_per_probe_dose(scan, prec, device="cuda")
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("spec", [w.ScanSpec(16, 16), w.ScanSpec(64, 64),
                                  w.ScanSpec(23, 19, order=w.RANDOM, seed=8, keep_fraction=0.7),
                                  w.ScanSpec(1, 1), w.ScanSpec(2, 1)])
def test_dose_full(cuda, spec):
    ref = oracle_dose(spec)
    g64 = gpu_dose(spec, "fp64")
    assert g64[0] == 0.0
    assert_fp64(g64, ref, "dose fp64")
    gm = gpu_dose(spec, "mixed")
    if len(ref) > 1:
        assert_mixed(gm[1:], ref[1:], ref.max(), "dose mixed")


@pytest.mark.parametrize("spec", [
    w.ScanSpec(12, 9, flyback_s=2.5e-6),
    w.ScanSpec(10, 10, order=w.SERPENTINE, flyback_s=4e-7, D_m2s=1e-12),
    w.ScanSpec(9, 9, order=w.RANDOM, seed=12,
               dwell_per_visit=10 ** np.random.default_rng(1).uniform(-7, -5, 81)),
])
def test_dose_general_timing(cuda, spec):
    ref = oracle_dose(spec)
    g64 = gpu_dose(spec, "fp64")
    assert g64[0] == 0.0
    assert_fp64(g64, ref, "general dose fp64")
    gm = gpu_dose(spec, "mixed")
    assert_mixed(gm[1:], ref[1:], ref.max(), "general dose mixed")
