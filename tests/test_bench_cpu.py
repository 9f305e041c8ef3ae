"""Host-side logic of bench.py, on the CPU: names, work counts and roofline arithmetic."""
import builtins
import os
import symtable

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def undefined_globals(path):
    """Global names referenced in a module but bound nowhere in it (nor builtins)."""
    src = open(path).read()
    top = symtable.symtable(src, path, "exec")
    bound = {s.get_name() for s in top.get_symbols() if s.is_assigned() or s.is_imported()}
    bound |= set(dir(builtins)) | {"__file__", "__name__", "__doc__", "__spec__", "__path__"}
    missing = set()

    def walk(t):
        for s in t.get_symbols():
            glob = t.get_type() == "module" or s.is_global()
            if glob and s.is_referenced() and s.get_name() not in bound:
                missing.add(s.get_name())
        for c in t.get_children():
            walk(c)

    walk(top)
    return missing


@pytest.mark.parametrize("name", ["bench.py", "__graft_entry__.py"])
def test_no_undefined_globals(name):
    assert undefined_globals(os.path.join(ROOT, name)) == set()


def test_checker_catches_a_missing_name(tmp_path):
    p = tmp_path / "m.py"
    p.write_text("def f():\n    return g(1)\n")
    assert undefined_globals(str(p)) == {"g"}


def test_work_counts():
    # FP64 algorithmic flops per (m, l, ring-pair) step: recursion + 2 real FMAs
    # per complex output and component (spin: 4 complex outputs per E/B pair)
    assert bench.flops_per_triple(0, 1) == 7 and bench.flops_per_triple(2, 1) == 26
    assert bench.flops_per_triple(2, 3) == 10 + 48
    # double-float FP32-pipe ops: compensated multiply-add 12, recursion 24 / 67
    assert bench.f32_ops_per_triple(0, 1) == 48 and bench.f32_ops_per_triple(2, 1) == 163
    assert bench.launches_per_step(2, "fp64") == 6 and bench.launches_per_step(0, "fp64") == 5
    assert bench.launches_per_step(0, "mixed") == 6
    assert bench.launches_per_step(2, "mixed", True) == 9 and bench.launches_per_step(0, "mixed", True) == 8


class _Plan:
    def triples(self, flags=0):
        return 10 ** 10

    def triples_joined(self):
        return 9 * 10 ** 9


def test_roofline_arithmetic(monkeypatch):
    stages = {"legendre_synthesis": (300.0, 3), "legendre_analysis": (450.0, 3)}
    peaks = {"sm_max_mhz": 2000.0}
    r = bench.roofline_for(stages, _Plan(), 2, "fp64", peaks, 3)
    assert r["kernel"] == "legendre_analysis" and r["ms_per_launch"] == pytest.approx(150.0)
    assert r["achieved"] == pytest.approx(26e10 / 0.150 / 1e12)
    assert r["peak"] == pytest.approx(152 * 4 * 2e9 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    # mixed form: the method's 26 flops per triple against the FP32 pipe's FMA-flop
    # rate; the double-float issue rate is a separate field
    m = bench.roofline_for(stages, _Plan(), 2, "mixed", peaks, 3)
    assert m["achieved"] == pytest.approx(26e10 / 0.150 / 1e12)
    assert m["peak"] == pytest.approx(152 * 128 * 2 * 2e9 / 1e12)
    assert m["frac"] == pytest.approx(m["achieved"] / m["peak"])
    assert m["issue_frac"] == pytest.approx(163e10 / 0.150 / 1e12 / (152 * 128 * 2e9 / 1e12))
    # the same work counted on the steps left after the join records
    assert m["triples_after_join"] == 9 * 10 ** 9
    assert m["frac_after_join"] == pytest.approx(0.9 * m["frac"])
    # with the box's measured pipe rates the peak is 2 x the measured FFMA rate
    peaks["pipes_measured"] = {"fp64_fma_tflops": 1.25, "fp32_fma_tops": 38.3, "fp32_add_tops": 38.3}
    m = bench.roofline_for(stages, _Plan(), 2, "mixed", peaks, 3)
    assert m["peak"] == pytest.approx(76.6) and m["frac"] == pytest.approx(26e10 / 0.150 / 1e12 / 76.6)
    assert bench.roofline_for(stages, _Plan(), 2, "fp64", peaks, 3)["peak"] == pytest.approx(1.25)
    # traffic: only while the kernel source still hashes as recorded
    monkeypatch.setattr(bench, "MEASURED_TRAFFIC", {"mixed:legendre_analysis": {"bytes": 123, "sha256": "0" * 64}})
    assert bench.roofline_for(stages, _Plan(), 2, "mixed", peaks, 3)["traffic"] is None


def test_headline_config_exceeds_l2():
    bench.set_workload(4095)
    assert bench.CONFIG["lmax"] == 4095 and bench.CONFIG["nlon"] == 8191
    assert bench.CONFIG["l2_policy"].startswith("inputs larger than L2")


def test_oracle_single_core_leg():
    # the cpu_baseline leg times the oracle on one core in a process of its own
    assert bench.oracle_single_thread_small() > 0


def test_fixed_oracle_sample_and_reference_line():
    # both arms time the same sample: 2 rings and 2 m values per core, poles and
    # both ends of the m range included; the reference arm prints its line with
    # the per-unit costs and the extrapolation formula
    import json
    import subprocess
    import sys

    bench.set_workload(4095)
    rsel, msel = bench.oracle_sample_sizes(16)
    assert len(rsel) == 32 and rsel[0] == 0 and rsel[-1] == 4095
    assert len(msel) == 32 and msel[0] == 0 and msel[-1] == 4095
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--lmax", "31", "--steps", "2",
                        "--warmup", "1"], cwd=bench.ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    cb = line["cpu_baseline"]
    assert line["impl"] == "reference" and line["value"] > 0 and len(cb["step_values_ms"]) == 2
    assert cb["value"] == line["value"]
    # the last step's value is the formula applied to its per-unit costs (32 rings, 32 m at lmax 31)
    t = cb["ms_per_ring_synthesis"] * 32 + cb["ms_per_m_analysis"] * 32
    assert abs(t - cb["step_values_ms"][-1]) <= 1e-9 * t
