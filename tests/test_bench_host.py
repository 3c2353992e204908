"""Host logic of bench.py (no GPU): the algorithmic byte count against the
hand count for the 27-point stencil 100^3 in beta(4,8), the plan labels,
the comment-insensitive kernel source hash and the parsing of the committed
ncu DRAM table it guards."""
from __future__ import annotations

import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _info(**kw):
    base = dict(nrows=10**6, ncols=10**6, nnz=26_463_592, nblocks=2_220_100, npanels=250_000,
                mask_bytes=4, value_dtype=0, flat=0, lanes_per_row=1)
    base.update(kw)
    return base


def test_algorithmic_bytes_of_the_27_point_stencil_in_beta_4_8(bench):
    # 8 B per value, 4 B column + 4 B mask per block, 8 B per panel pointer
    # pair, x and y in FP64: 211.7 + 8.9 + 8.9 + 2.0 + 8.0 + 8.0 = 247.5 MB
    b = bench.algorithmic_bytes(_info())
    assert b == 8 * 26_463_592 + 8 * 2_220_100 + 8 * 250_001 + 16 * 10**6
    assert b / 1e6 == pytest.approx(247.5, abs=0.05)


def test_reduced_precision_bytes_use_fp32_vectors(bench):
    f32 = bench.algorithmic_bytes(_info(value_dtype=1))
    bf16 = bench.algorithmic_bytes(_info(value_dtype=2))
    fp64 = bench.algorithmic_bytes(_info())
    assert fp64 - f32 == 4 * 26_463_592 + 8 * 10**6
    assert f32 - bf16 == 2 * 26_463_592


def test_plan_labels(bench):
    assert bench.plan_label(_info(flat=1)) == "blocks"
    assert bench.plan_label(_info(flat=2)) == "expanded"
    assert bench.plan_label(_info(flat=3)) == "values"
    assert bench.plan_label(_info(flat=0, lanes_per_row=4)) == "rows/G4"
    assert bench.plan_label(_info(flat=0, lanes_per_row=1, body=2, dynamic=1)) == "rows/G1/b2/dyn"
    assert bench.plan_label(_info(flat=0, lanes_per_row=2, body=0, dynamic=0)) == "rows/G2/b0"
    assert bench.plan_label(_info(flat=0, lanes_per_row=1, body=7, dynamic=1)) == "rows/G1/b7/dyn"


def test_source_hash_ignores_comments_only(bench, tmp_path, monkeypatch):
    csrc = os.path.join(ROOT, "paper_2307_14774_gb300", "csrc")
    text = open(os.path.join(csrc, "spc5_spmv.cu")).read()
    flat = open(os.path.join(csrc, "spc5_flat.cuh")).read()
    fake = tmp_path / "paper_2307_14774_gb300" / "csrc"
    fake.mkdir(parents=True)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (fake / "spc5_spmv.cu").write_text(text)
    (fake / "spc5_flat.cuh").write_text(flat)
    h0 = bench.kernel_source_hash()
    (fake / "spc5_spmv.cu").write_text("// a new comment\n" + text.replace("\n\n", "\n\n\n", 3))
    assert bench.kernel_source_hash() == h0
    (fake / "spc5_spmv.cu").write_text(text.replace("kVRound = 256", "kVRound = 128", 1))
    assert bench.kernel_source_hash() != h0
    (fake / "spc5_spmv.cu").write_text(text)
    (fake / "spc5_flat.cuh").write_text(flat.replace("kFlatKB = 4", "kFlatKB = 8", 1))
    assert bench.kernel_source_hash() != h0


def test_dram_ratio_table_parses_and_is_guarded_by_the_source_hash(bench, tmp_path,
                                                                  monkeypatch):
    """profiles/spc5_spmv_dram.txt holds, per benchmark case, the ncu DRAM
    bytes of one launch on the profile-scale instance, its algorithmic bytes
    and their ratio; bench.py applies the ratio only while the table's source
    hash is the kernels' (else the roofline's traffic is null)."""
    prof = tmp_path / "profiles"
    prof.mkdir()
    rows = ["# matrix beta dram_bytes algorithmic_bytes ratio", "source_sha256: abcd"]
    rows += [f"{m} {r}x{c} 1000 900 {1000 / 900:.4f}" for m in bench.MATRICES
             for r, c in bench.BETAS]
    (prof / "spc5_spmv_dram.txt").write_text("\n".join(rows) + "\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "abcd")
    table = bench.ncu_traffic_ratios()
    assert set(table) == {(m, f"{r}x{c}") for m in bench.MATRICES for r, c in bench.BETAS}
    assert all(v == pytest.approx(1000 / 900, abs=1e-4) for v in table.values())
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.ncu_traffic_ratios() is None


def test_committed_dram_table_if_present_covers_every_case(bench, monkeypatch):
    path = os.path.join(ROOT, "profiles", "spc5_spmv_dram.txt")
    if not os.path.exists(path):
        pytest.skip("no committed DRAM table")
    stored = [ln.split(":", 1)[1].strip() for ln in open(path) if ln.startswith("source_sha256:")]
    assert len(stored) == 1
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: stored[0])
    table = bench.ncu_traffic_ratios()
    assert table and all(0.5 < v < 3.0 for v in table.values())


def test_err_over_tol(bench):
    import numpy as np
    y_ref = np.array([1.0, 2.0, 0.0, 5.0])
    scale = np.array([10.0, 20.0, 0.0, 1.0])
    y = y_ref + np.array([1e-13, -1e-12, 0.0, 0.0])
    assert bench.err_over_tol(y, y_ref, scale, 1e-13) == pytest.approx(0.5, rel=1e-3)
    y[2] = 1e-300  # an error on a row whose scale is zero
    assert bench.err_over_tol(y, y_ref, scale, 1e-13) == float("inf")


def test_roofline_reports_the_longest_launch_against_hbm(bench):
    rows = [{"matrix": "stencil27", "beta": "4x8", "us": 50.0, "bytes": 247_500_000,
             "nnz": 26_463_592, "plan": "rows/G1"},
            {"matrix": "fem3d", "beta": "4x8", "us": 600.0, "bytes": 2_092_500_000,
             "nnz": 238_367_592, "plan": "rows/G1"}]
    ro = bench.roofline_object(rows, 6687.5, "measured", 1.25, "measured",
                               {("fem3d", "4x8"): 1.05}, {"frac": 0.5})
    assert ro["bound"] == "hbm" and ro["unit"] == "GB/s"
    assert ro["kernel"].startswith("FP64 SpMV fem3d beta(4x8)")
    assert ro["achieved"] == pytest.approx(2_092_500_000 / 600e-6 / 1e9, rel=1e-3)
    assert ro["frac"] == pytest.approx(ro["achieved"] / 6687.5, rel=1e-3)
    assert ro["traffic"] == pytest.approx(1.05 * 2_092_500_000, rel=1e-6)
    assert ro["fp64_pipe"]["frac"] == pytest.approx(2 * 238_367_592 / 600e-6 / 1e12 / 1.25,
                                                    rel=1e-3)


def test_cpu_baseline_references_do_not_depend_on_the_thread_count(bench):
    """The OpenMP build of the oracle, timed by the CPU baseline, gives the
    same products bit for bit as the single-threaded oracle the tests use."""
    import numpy as np

    import oracle
    import synth
    hosts = {"a": (synth.powerlaw(3000, seed=5), None), "b": (synth.fem3d(500, seed=1), None)}
    hosts = {k: (A, synth.vector_uniform(A.ncols, seed=2)) for k, (A, _) in hosts.items()}
    rec, refs = bench.cpu_baseline(hosts, lambda m: None, reps=1)
    assert rec["oracle_all"]["gflops"] > 0 and rec["plain_one"]["threads"] == 1
    assert isinstance(rec["cpu_model"], str) and rec["cpu_model"]
    for name, (A, x) in hosts.items():
        y, s = oracle.csr_spmv(A, x)
        assert np.array_equal(refs[name][0], y) and np.array_equal(refs[name][1], s)
