"""Host-side pieces of bench.py: the algorithmic byte model behind the
roofline figures (pass by pass, against per-cell counts and the large box's
total), the equal-error interpolation, and the whole-job aggregation."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_fused_pass_model_per_cell():
    """Film 256x128x4 in FP32 (r = 4, complex c = 8 bytes): XF reads m (3r)
    and writes the packed half spectrum (3c) = 36 B/cell; XI the reverse;
    the fused YZ pass reads and writes the spectrum (6c = 48 B/cell) plus the
    tensor octant (nx+1)(Py/2+1)(Pz/2+1) x 6 components once."""
    n = (256, 128, 4)
    cells = 256 * 128 * 4
    m = bench.demag_pass_bytes(n, 4, split=False)
    assert m["x_forward_fft"] == 36 * cells
    assert m["x_inverse_fft"] == 36 * cells
    assert m["yz_fft_tensor_multiply"] == 48 * cells + 257 * 129 * 5 * 6 * 4
    # FP64 doubles every term
    m8 = bench.demag_pass_bytes(n, 8, split=False)
    assert all(m8[k] == 2 * m[k] for k in m)
    bm = bench.byte_model({"mesh": {"n": n}, "integrator": {"extrap_order": 4}}, 4)
    assert all(bm[k] == m[k] for k in m)


def test_stage_model_per_cell_dp54_p4():
    """DP54 with 4th-order extrapolation in FP32 (u = 12 B/cell): stage 1
    reads m0 and the exact field and writes F_1 and Y_2 (4u = 48 B); stages
    2..6 read Y_k, five history fields, the F_l with nonzero b and m0 and
    write two fields: 120, 132, 144, 156, 156 B (b72 = 0); DP54 is FSAL, so
    stage 6 also writes the new m and reads and writes the compensated
    state's low words in FP32: 156 + 36 = 192 B; the last stage reads Y_7,
    the history and F_l for l in {1, 3, 4, 5, 6} (c_2 = c_2 - c^_2 = 0) and
    writes F_7: 144 B."""
    cells = 256 * 128 * 4
    mean, last = bench.stage_bytes(cells, 4, 4)
    assert mean == pytest.approx((48 + 120 + 132 + 144 + 156 + 192) / 6 * cells)
    assert last == 144 * cells
    m8, last8 = bench.stage_bytes(cells, 8, 4)
    assert last8 == 2 * 144 * cells and m8 == pytest.approx(2 * (48 + 120 + 132 + 144 + 156 + 168) / 6 * cells)
    # FSAL: the last Eq. 4 row equals the Eq. 3 weights and c_7 = 0
    import oracle as O
    t = O.tableau("RKDP54")
    assert list(t["b"][6][:6]) == list(t["c"][:6]) and t["c"][6] == 0.0
    # the read pattern is the tableau's nonzero pattern (oracle's copy of the
    # published coefficients)
    import oracle as O
    t = O.tableau("RKDP54")
    for k, reads in bench.DP54_B_READ.items():
        assert reads == [l for l in range(k) if t["b"][k + 1][l] != 0.0]
    assert bench.DP54_LAST_READ == [l for l in range(6) if t["c"][l] != 0.0 or t["c"][l] != t["chat"][l]]


def test_split_pass_model_of_the_large_box():
    """512x512x16 FP32 with the split y-z passes: the y spectrum is Py/ny = 2
    times the packed half spectrum; one evaluation moves 1.41 GB, the figure
    the large-box roofline divides by the measured time."""
    n = (512, 512, 16)
    cells = 512 * 512 * 16
    m = bench.demag_pass_bytes(n, 4, split=True)
    assert m["x_forward_fft"] == 36 * cells
    # YF: spectrum in (3c/cell), y spectrum out (2 x 3c/cell); ZM: y spectrum in
    # and out + tensor; YI: y spectrum in, spectrum out
    yspec = 2 * 24 * cells
    tensor = 513 * 513 * 17 * 6 * 4
    assert m["yz_fft_tensor_multiply"] == (24 * cells + yspec) + (2 * yspec + tensor) + (yspec + 24 * cells)
    assert sum(m.values()) == pytest.approx(1.41e9, rel=0.01)
    # the full field (mmx_demag) also reads m in XI for the self term
    mf = bench.demag_pass_bytes(n, 4, split=True, self_term=True)
    assert mf["x_inverse_fft"] - m["x_inverse_fft"] == 12 * cells
    assert mf["x_forward_fft"] == m["x_forward_fft"]


def test_speed_at_error_interpolates_in_log_log():
    rows = [{"eps": 1e-5, "ns_per_s": 1.0}, {"eps": 1e-3, "ns_per_s": 4.0}, {"eps": 1e-4, "ns_per_s": 2.0}]
    assert bench.speed_at_error(rows, 1e-4) == (pytest.approx(2.0), True)        # a sweep point
    v, inside = bench.speed_at_error(rows, np.sqrt(1e-5 * 1e-4))                   # geometric midpoint
    assert inside and v == pytest.approx(np.sqrt(2.0))
    v, inside = bench.speed_at_error(rows, 1e-2)                                   # beyond: same slope
    assert not inside and v == pytest.approx(8.0)
    v, inside = bench.speed_at_error(rows, 1e-6)
    assert not inside and v == pytest.approx(0.5)


def test_aggregate_is_all_units_over_the_slowest_rank():
    value, t_max = bench.aggregate(0.2, 1.5, 4, lambda x: 2.0 * x, lambda x: 4.0 * x)
    assert t_max == 3.0 and value == pytest.approx(0.8 / 3.0)


def test_eps_time_is_eq7_over_time_samples():
    """bench.eps_time (the bench's own copy, no oracle import on the product
    path) equals the oracle's Eq. 7 over time samples of <m>."""
    import oracle as O
    rng = np.random.default_rng(3)
    a, b = rng.normal(size=(3, 40)), rng.normal(size=(3, 40))
    assert bench.eps_time(a, b) == pytest.approx(O.epsilon_time(a, b), rel=1e-14)
    assert bench.eps_time(a, a) == 0.0


def _row(sm, max_sm=2070, reasons=("Not Active",) * 4):
    return ["0", str(sm), str(max_sm), "900.0", "0x0"] + list(reasons)


def test_clock_sampler_keeps_the_timed_window():
    s = bench.ClockSampler(0, period_ms=50)
    s.rows = [(0.90, _row(1000)), (1.00, _row(2070)), (1.05, _row(2055)), (1.10, _row(2070)),
              (1.40, _row(1200, reasons=("Active", "Active", "Not Active", "Not Active")))]
    s.window = [0.99, 1.12]
    out = s.stop()
    assert out["samples"] == 3 and out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == []                     # the throttled sample lies outside the window


def test_clock_sampler_region_shorter_than_a_period():
    s = bench.ClockSampler(0, period_ms=200)
    s.rows = [(1.00, _row(2070)), (1.60, _row(2040, reasons=("Not Active",) * 3 + ("Active",)))]
    s.window = [1.05, 1.10]
    out = s.stop()
    assert out["samples"] == 0 and out["adjacent_samples"] == 2
    assert out["sm_mhz"] == 2055.0 and out["reasons"] == ["sw_power_cap"]
