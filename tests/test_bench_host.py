"""Host logic of bench.py on CPU: the clock record that decides whether a
measurement is kept (median SM clock, throttle reasons from nvidia-smi's
CSV), and the closed-form work counts behind the roofline numbers."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
import bench                                # noqa: E402


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.proc = _FakeProc()
    s.lines = list(lines)
    return s


def test_clock_record_median_and_reasons():
    # index, clocks.sm, clocks.max.sm, power, active, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 1980, 2070, 1390.2, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 2010, 2070, 1201.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "garbage line",
             "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    rec = _sampler(lines).stop()
    assert rec["samples"] == 3
    assert rec["sm_mhz"] == 2010.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]


def test_clock_record_flags_thermal_and_hw_slowdown():
    lines = ["0, 1500, 2070, 1000, 0x48, Active, Not Active, Active, Not Active"] * 3
    rec = _sampler(lines).stop()
    assert rec["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_record_without_nvidia_smi():
    s = bench.ClockSampler(0)
    assert s.stop() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}


def test_sweep_work_counts():
    """Per-unit counts of a correction-sweep launch: FP64 flops (SIPG
    application 8(P+1)+20 per DOF; convective per node 4(P+1) per component
    plus the flux (Burgers: 4 per node, 20 per face node on 4(P+1) of the
    (P+1)^2 nodes); CG iteration 10 more, right-hand side 12, quadrature 2M;
    two SIPG and two convective applications and two right-hand sides per
    SI(2) node) and bytes (19 FP64 arrays per node, 11 per CG iteration)."""
    P, nc, M, nv = 7, 2, 5, 131072
    mv, cv = 8 * 8 + 20, (2 * 4 * 8 + 4 + 4 * 20 / 8) / 2
    per_node = 2 * mv + 2 * cv + 2 * 12 + 2 * M
    assert bench.sweep_flops(P, nc, M, 1, 0, nv, "burgers") == nv * M * per_node
    assert (bench.sweep_flops(P, nc, M, 1, 10, nv, "burgers") - bench.sweep_flops(P, nc, M, 1, 0, nv, "burgers")
            == nv * 10 * (mv + 10))
    # one component: the convective count is per node
    assert bench.conv_flops_per_dof(8, 1, "convdiff") == 4 * 9 + 2 + 4 * 8 / 9
    # a system's derivative sums scale with the components, its flux per node does not
    assert bench.conv_flops_per_dof(7, 4, "euler") == 4 * 8 + (24 + 4 * 60 / 8) / 4
    assert bench.sweep_bytes(M, 1, 0, nv) == 8 * nv * M * 19
    assert bench.sweep_bytes(M, 1, 3, nv) - bench.sweep_bytes(M, 1, 0, nv) == 8 * nv * 3 * 11


def test_mlp_flop_counts():
    """Forward: three products (n_in x H, H x H, H x q per row); training adds
    the five backward products (three weight gradients, two input gradients)."""
    fwd, train = bench.mlp_flops(10, 325, 112, 36)
    assert fwd == 2 * 10 * (325 * 112 + 112 * 112 + 112 * 36)
    assert train - fwd == 2 * 10 * (325 * 112 + 2 * 112 * 112 + 2 * 112 * 36)


def test_whole_job_value_weak_scaling():
    assert bench.whole_job_value(1000.0, 10, 1, 2.0) == 1000.0 * 10 / 2e-3
    assert bench.whole_job_value(1000.0, 10, 4, 2.0) == 4 * bench.whole_job_value(1000.0, 10, 1, 2.0)


def test_converged_count_ten_percent_rule():
    """errs[k] = error after k+1 iterations; converged at the first count
    after which one more iteration changes the error by less than 10 %."""
    assert bench.converged_count([1.0, 0.5, 0.46, 0.45]) == 2
    assert bench.converged_count([1.0, 0.95]) == 1
    assert bench.converged_count([1.0, 0.5, 0.2]) is None


def test_oracle_sample_grid_bounded():
    """Workloads whose fine level exceeds the CPU baseline's size bound are
    sampled on a coarser element grid of the same physics."""
    import argparse
    a = argparse.Namespace(workload="euler256", small=False, oracle_nel=0)
    assert bench.oracle_nel_for(a) == 64
    a = argparse.Namespace(workload="burgers2d", small=False, oracle_nel=0)
    assert bench.oracle_nel_for(a) == 0


def test_kernel_digest_tracks_sources():
    d1 = bench.kernel_digest(bench.ENS_KERNEL_SOURCES)
    assert d1 == bench.kernel_digest(bench.ENS_KERNEL_SOURCES) and len(d1) == 16
    assert d1 != bench.kernel_digest(bench.SWEEP_KERNEL_SOURCES)


def test_burgers_front_variants_are_valid_level_lists():
    """Every variant of the shock-capturing arm's front table: levels coarse to
    fine, element grids equal or 2:1, degrees and node counts non-decreasing,
    the finest level the paper's 40 elements of degree 8 with 7 nodes."""
    for name, levels, start in bench.BURGERS_FRONT_VARIANTS:
        assert levels[-1] == (40, 8, 7), name
        assert (start is None) == (len(levels) == 1), name
        for (n0, p0, m0), (n1, p1, m1) in zip(levels, levels[1:]):
            assert n1 in (n0, 2 * n0) and p1 >= p0 and m1 >= m0, name
