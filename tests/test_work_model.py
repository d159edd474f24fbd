"""The benchmark's work model (the numerator of its roofline fraction) and its clock record,
pinned on the CPU.

A float-float Lanczos step is charged for the line transforms the library runs on the pruned
box (z-sticks through the sphere, y-columns on the x values that hold sticks, x-rows of every
plane, each once forward and once back), the potential product, and the projector dots and
updates.  These tests pin the model against independent counts: the stick and column counts of
the 64-atom supercell against the oracle's own sphere enumeration, the textbook twiddle count
of a radix-4 16-point transform, and a hand tally of the prime-factor 72-point and 36-point
transforms."""
import numpy as np

import bench
import instances.generate as G
import oracle as O


class _Supercell:
    fft_dims = (72, 72, 72)
    kb_atom = np.zeros(64, dtype=np.int32)
    n_occ = 128


def _supercell_plan():
    a, _ = G.supercell64_cell()
    mil, _ = O.gsphere(a, (0.0, 0.0, 0.0), 25.0)
    return bench.plan_info(_Supercell, mil)


def test_supercell_pruned_box_lines():
    """18 277 plane waves at Gamma fill 845 z-sticks, which sit on 33 distinct x values; a step
    transforms 2 x (845 + 72 x 33 + 72 x 72) = 16 810 lines of 72 points."""
    p = _supercell_plan()
    assert p["npw"] == 18277
    assert p["nstick"] == 845 and p["nxcol"] == 33
    lines = bench.apply_line_counts(p)
    assert [n for n, _ in lines] == [72, 72, 72]
    assert sum(c for _, c in lines) == 2 * (845 + 72 * 33 + 72 * 72) == 16810


def test_radix4_line_textbook_count():
    """16 points in two radix-4 stages: 2 x 4 butterflies of 8 complex additions, and
    (16/4 - 1) x 3 = 9 non-trivial twiddle multiplications (none in the last stage)."""
    assert bench.fft_line_ops(16) == (64, 9, 0)


def test_prime_factor_lines_hand_tally():
    """72 = 8 x 9 with no twiddles between the two stages.  An 8-point DFT = two 4-point
    (8 additions each) + four 2-point (2 each) + (2 - 1)(4 - 1) = 3 inner twiddles: 24 additions,
    3 multiplications.  A 9-point DFT = six 3-point DFTs (6 additions, 2 real scalings each) +
    (3 - 1)(3 - 1) = 4 inner twiddles: 36 additions, 4 multiplications, 12 scalings.  A line is
    9 eight-point + 8 nine-point DFTs: 504 additions, 59 multiplications, 96 scalings; 36 = 4 x 9:
    9 four-point + 4 nine-point: 216, 16, 48."""
    assert bench.fft_line_ops(72) == (9 * 24 + 8 * 36, 9 * 3 + 8 * 4, 8 * 12)
    assert bench.fft_line_ops(36) == (9 * 8 + 4 * 36, 4 * 4, 4 * 12)


def test_supercell_step_operations():
    """The float-float step: 16 810 lines at 22 / 38 / 14 FP32 operations per complex addition /
    multiplication / real scaling, 14 per potential sample of the 72^3 box, and 120 per plane
    wave and projector row (dot and update, 60 each) plus 300 per plane wave: 678.5 M."""
    p = _supercell_plan()
    per_line = 22 * 504 + 38 * 59 + 14 * 96
    expect = 16810 * per_line + 14 * 72 ** 3 + 18277 * (120 * (128 + 64) + 300)
    assert bench.step_df32_ops(p) == expect
    assert abs(expect - 678.48e6) < 0.01e6


def test_clock_samples_parsing():
    """The clock record of the timed region: median SM clock, the maximum, and every throttle
    reason reported Active in any sample (Not Active ignored; malformed lines skipped)."""
    lines = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2055, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "[N/A]",
        "0, [N/A], 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    c = bench.parse_clocks(lines)
    assert c == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    c = bench.parse_clocks(lines[:1] + ["0, 1500, 2070, 1000, 0x8, Active, Not Active, Active, Not Active"])
    assert c["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"] and c["sm_mhz"] == 1785.0
    assert bench.parse_clocks([])["sm_mhz"] is None
