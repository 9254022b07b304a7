"""Host-side checks of the benchmark contract (no GPU): the reference arm's JSON line carries every key
the contract asks for, and the committed ncu traffic figure is used only on the kernel source it was
measured on."""
import argparse
import hashlib
import json
import os
import re

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _args(**kw):
    base = dict(gpus=1, steps=2, warmup=1, impl="reference", nshot=100, nt=4000, segment=0)
    base.update(kw)
    return argparse.Namespace(**base)


def test_reference_line_has_the_contract_keys(monkeypatch, capsys):
    calls = []

    def fake_sample(wl, nt_sample, nshot_sample, threads):
        calls.append((nt_sample, nshot_sample, threads))
        return 0.25, 1.5, f"{nshot_sample} shots x nt={nt_sample} of the {wl.name} grid (B~ + B~*)"

    monkeypatch.setattr(bench, "oracle_sample", fake_sample)
    monkeypatch.delenv("RANK", raising=False)
    bench.run_reference(_args())
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert len(calls) == 3                                  # warmup + steps samples
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] == pytest.approx(0.25) and line["ms_per_step"] == pytest.approx(1500.0)
    assert line["higher_is_better"] is True and line["vs_baseline"] is None
    assert line["config"]["workload"].startswith("marmousi2-like")
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_is_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setattr(bench, "oracle_sample", lambda *a: pytest.fail("a non-zero rank ran the oracle"))
    monkeypatch.setenv("RANK", "1")
    bench.run_reference(_args())
    assert capsys.readouterr().out == ""


def test_traffic_figure_only_for_the_measured_kernel_source():
    src = os.path.join(ROOT, "paper_2206_02362_gb300", "csrc", "k_prop.cu")
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    txt = open(os.path.join(ROOT, "profiles", "k_prop_marmousi2_ncu.md")).read()
    m = re.search(r"k_prop\.cu sha256\[:16\]:\s*([0-9a-f]{16})", txt)
    assert m, "the summary names the source it was taken on"
    t = bench.ncu_traffic()
    if m.group(1) != h:
        assert t is None
    else:
        assert t is not None
        ratio = t["dram_bytes_per_launch"] / t["algorithmic_bytes_per_launch"]
        assert 0.9 < ratio < 1.2


def test_updates_per_step_counts_four_propagations():
    wl = bench.workload(_args())
    NZ, NX = wl.padded
    assert bench.updates_per_step(wl) == pytest.approx(4.0 * wl.nshot * NZ * NX * (wl.nt - 1))
