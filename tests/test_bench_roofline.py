"""The roofline accounting of bench.py on CPU: a pass's SM clocks per pair are
max(fp32 / 128, mufu / 16) of its form, and the GB pass mixes its far and
full forms by the share of pairs with D >= 18."""
import pytest

import bench


def test_single_form_clocks():
    assert bench.clk_per_pair_per_sm(24, 1) == pytest.approx(24 / 128)
    assert bench.clk_per_pair_per_sm(8, 4) == pytest.approx(4 / 16)  # MUFU-bound form
    for name in ("born", "chain"):
        assert bench.pass_clk(name, 0.7) == bench.clk_per_pair_per_sm(*bench.PASS_COST[name])


def test_gb_mix_interpolates_its_two_forms():
    full = bench.clk_per_pair_per_sm(*bench.PASS_COST["gb"])
    far = bench.clk_per_pair_per_sm(*bench.GB_FAR_COST)
    assert far < full
    assert bench.pass_clk("gb", 0.0) == pytest.approx(full)
    assert bench.pass_clk("gb", 1.0) == pytest.approx(far)
    assert bench.pass_clk("gb", 0.25) == pytest.approx(0.25 * far + 0.75 * full)


def test_far_forms_cost_less_in_both_directions():
    assert all(a <= b for a, b in zip(bench.GB_FAR_COST, bench.PASS_COST["gb"]))
    assert all(a <= b for a, b in zip(bench.BACKWARD_FAR_COST, bench.BACKWARD_COST))
    # the backward totals are the sums of their three passes' forms
    assert bench.BACKWARD_COST[0] == bench.PASS_COST["born"][0] + 32 + 45
    assert bench.BACKWARD_FAR_COST[0] == bench.PASS_COST["born"][0] + 22 + 45


@pytest.mark.parametrize("steps,warmup", [(20, 5), (100, 5), (200, 3), (7, 3), (199, 5), (150, 10)])
def test_timed_window_holds_the_schedule_events(steps, warmup):
    """The window leaves room for the warm-up steps after step 0, holds an
    exchange step, and holds MC steps in their proportion (one per 10 steps,
    give or take the ends); whole periods when K is a multiple of 100."""
    first = bench.window_start(steps, warmup)
    assert first - warmup >= 1
    ev = bench.schedule_events(first, steps)
    assert ev["last_step"] - ev["first_step"] + 1 == steps
    assert ev["exchange_steps"] >= 1
    assert abs(ev["mc_ph_steps"] - steps / 10) <= 1
    if steps % 100 == 0:
        assert ev["exchange_steps"] == steps // 100 and ev["mc_ph_steps"] == steps // 10


def test_schedule_launches_counts_the_launch_list():
    """The kernels of one step as the launch list of the 384-walker workload
    shows them: 12 per plain step; +6 at an MC step with both kinds; +2 more
    at an exchange step."""
    assert bench.schedule_launches(91) == 12
    assert bench.schedule_launches(110) == 18
    assert bench.schedule_launches(100) == 20
    assert sum(bench.schedule_launches(t) for t in range(91, 111)) == 20 * 12 + 12 + 2
