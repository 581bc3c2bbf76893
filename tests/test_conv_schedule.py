"""Schedule of the tensor-memory convolution (surrogate, host-side check of its index rules).

The persistent kernel walks segments of kSeg output rows of a dilation-strided chain
(rows rho, rho + d, rho + 2d, ... of one 128-pixel column strip) and keeps input rows in a
ring of four slots: chain row i sits in slot i mod 4, output row j reads chain rows j - 1,
j, j + 1, and while row j's MMAs run the kernel copies in chain row j + 2.  This test
restates those rules (the segment length is read from the kernel source) and checks, for
every row count and dilation the surrogate uses or the tests exercise, that every output
row is produced exactly once, that every MMA finds its three input rows in their slots,
and that no copy overwrites a slot an MMA in flight is reading.
"""
import os
import re

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_2507_00294_gb300", "csrc", "dd_surrogate.cu")


def seg_len():
    m = re.search(r"constexpr int kSeg = (\d+);", open(SRC).read())
    assert m, "segment length not found in the kernel source"
    return int(m.group(1))


def items(H, dil, k_seg):
    out = []
    for rho in range(dil):
        J = (H - rho + dil - 1) // dil
        for s in range((J + k_seg - 1) // k_seg):
            j0 = s * k_seg
            out.append((rho, j0, min(J, j0 + k_seg)))
    return out


def test_ring_schedule_covers_rows_and_never_overwrites_live_slots():
    k_seg = seg_len()
    for H in (1, 2, 7, 24, 36, 40, 128):
        for dil in range(1, 33):
            rows = []
            for rho, j0, j1 in items(H, dil, k_seg):
                slot = {}
                for i in range(j0 - 1, j0 + 2):
                    slot[(i + 4) & 3] = i

                def mma(j):
                    for ky in range(3):
                        assert slot[(j + 3 + ky) & 3] == j + ky - 1, (H, dil, rho, j, ky)
                    return {(j + 3 + ky) & 3 for ky in range(3)}

                inflight = mma(j0)
                for j in range(j0, j1):
                    if j + 1 < j1:
                        s_new = (j + 2) & 3
                        assert s_new not in inflight, (H, dil, j)
                        slot[s_new] = j + 2
                    rows.append(rho + j * dil)
                    inflight = mma(j + 1) if j + 1 < j1 else set()
            assert sorted(rows) == list(range(H)), (H, dil)
