"""The unit-count roofline bench.py reports for its ALU-bound kernels (CPU).

Per SM and clock a GB300 issues 4 x 32 lane instructions and 16 MUFU lane
operations; a kernel's peak pairs/s is the tighter of the two limits for its
per-pair counts.  These checks pin the arithmetic and which limit binds for
each kernel at 152 SMs and 2.07 GHz (the figures DESIGN's measurement table
quotes), so that a change to a count shows up here."""
import pytest

import bench

SM, CLK = 152, 2.07e9


def test_issue_and_mufu_limits_by_hand():
    peak, limiter = bench.alu_roofline("rsi", SM, CLK, {"fp32": 100.0, "mufu": 1.0, "lds": 0.0})
    assert limiter == "issue"
    assert peak == pytest.approx(128 * SM * CLK / 101.0)
    peak, limiter = bench.alu_roofline("rsi", SM, CLK, {"fp32": 1.0, "mufu": 4.0, "lds": 0.0})
    assert limiter == "mufu"
    assert peak == pytest.approx(16 * SM * CLK / 4.0)


@pytest.mark.parametrize("kind,gpair", [("rsi", 1678.08), ("piston", 1678.08)])
def test_single_frequency_kernels_are_mufu_bound(kind, gpair):
    """3 MUFU per pair (rsqrt, sin, cos): 16 x 152 x 2.07e9 / 3 pairs/s."""
    peak, limiter = bench.alu_roofline(kind, SM, CLK)
    assert limiter == "mufu"
    assert peak / 1e9 == pytest.approx(gpair, rel=1e-6)


def test_multi_frequency_counts():
    """nf frequencies on shared points: 2 + 1/nf MUFU per pair-term; at
    nf = 3 the RSI kernel's bound is 2158 Gpair-terms/s."""
    ops = bench.multi_ops("rsi", 3)
    assert ops["mufu"] == pytest.approx(2.0 + 1.0 / 3)
    assert ops["fp32"] == pytest.approx(14.0 / 6 + 4.5)
    assert ops["lds"] == pytest.approx(5.0 / 6)  # geometry 2 float4 + 1 per frequency, per source pair
    peak, limiter = bench.alu_roofline("rsi", SM, CLK, ops)
    assert limiter == "mufu"
    assert peak / 1e9 == pytest.approx(2157.53, rel=1e-5)
    for nf in (2, 3, 4):  # sharing the geometry never raises the MUFU work per pair-term
        assert bench.multi_ops("rsi", nf)["mufu"] < bench.OPS["rsi"]["mufu"]


def test_shared_harmonic_counts_move_the_rsi_bound_to_the_fp32_pipe():
    """Three frequencies with one formed from another by the double angle: 5
    MUFU per pair (rsqrt and two sincos) against 44 FP32-pipe lane cycles for
    RSI, so the FP32 pipe binds at 128 / 44 pairs per SM clock, 2.91 pairs per
    clock where the plain three-frequency kernel's MUFU allowed 2.29; the
    piston stays MUFU-bound at 16 / 5."""
    ops = bench.multi_ops("rsi", 3, harmonic=True)
    assert ops["mufu"] * 3 == pytest.approx(5.0)
    assert ops["fma_pipe"] * 3 == pytest.approx(44.0)
    peak, limiter = bench.alu_roofline("rsi", SM, CLK, ops)
    assert limiter == "fma"
    assert peak == pytest.approx(128 * SM * CLK / ops["fma_pipe"])
    plain, _ = bench.alu_roofline("rsi", SM, CLK, bench.multi_ops("rsi", 3))
    assert peak / plain == pytest.approx((128 / 44) / (16 / 7), rel=1e-9)
    pk, plim = bench.alu_roofline("piston", SM, CLK, bench.multi_ops("piston", 3, harmonic=True))
    assert plim == "mufu" and pk == pytest.approx(16 * SM * CLK * 3 / 5)


def test_ray_tracing_counts_include_compares_and_bind_on_the_fp32_pipe():
    """The packed ray-tracing pair with one Newton step: 11 MUFU against 102
    FP32-pipe lane cycles (the path differences by a Newton step and T12
    folded into the amplitude's reciprocal square root moved work from the
    MUFU to the FP32 pipe), so the FP32 pipe binds, ahead of the MUFU and of
    issue; the compares, selects and clamps (the "alu" count) take issue
    slots too."""
    o = bench.OPS["raytrace"]
    peak, limiter = bench.alu_roofline("raytrace", SM, CLK)
    assert limiter == "fma"
    assert peak / 1e9 == pytest.approx(128 * SM * CLK / o["fma_pipe"] / 1e9)
    assert o["fma_pipe"] / 128 > o["mufu"] / 16
    no_alu = dict(o, alu=0)
    issue_with = (o["fp32"] + o["alu"] + o["mufu"] + o["lds"]) / (128 * SM * CLK)
    issue_without = (no_alu["fp32"] + no_alu["mufu"] + no_alu["lds"]) / (128 * SM * CLK)
    assert issue_with > issue_without
    assert o["fma_pipe"] / 128 > issue_with * SM * CLK


def test_unpacked_rsi_kernel_was_issue_bound():
    """The unpacked RSI kernel's 23 FP32 + 3 MUFU + 1 LDS = 27 slots per pair:
    issue-bound at 128 x 152 x 2.07e9 / 27 = 1492 Gpair/s (the variant-2 row)."""
    peak, limiter = bench.alu_roofline("rsi", SM, CLK, {"fp32": 23.0, "mufu": 3.0, "lds": 1.0})
    assert limiter == "issue"
    assert peak / 1e9 == pytest.approx(1491.7, rel=1e-3)


def test_fma_pipe_limit():
    """The FP32 pipe does 128 FMA lanes per SM per clock and a packed f32x2
    instruction occupies it two cycles: a kernel of 30 packed instructions
    per pair is FP32-pipe bound at 128 x 152 x 2.07e9 / 60 pairs/s though it
    issues only 30 instructions."""
    peak, limiter = bench.alu_roofline("rsi", SM, CLK, {"fp32": 30.0, "mufu": 1.0, "lds": 0.0, "fma_pipe": 60.0})
    assert limiter == "fma"
    assert peak == pytest.approx(128 * SM * CLK / 60.0)
    # the packed single-frequency RSI kernel in its polar form leaves the MUFU
    # the clear limiter: 19/128 of a clock per pair on the FP32 pipe against
    # the MUFU's 3/16 (the Cartesian form's 23/128 co-limited the two)
    o = bench.OPS["rsi"]
    assert o["fma_pipe"] / 128 < 0.8 * o["mufu"] / 16
    assert bench.alu_roofline("rsi", SM, CLK)[1] == "mufu"
