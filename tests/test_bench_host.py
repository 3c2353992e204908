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


def test_source_hash_ignores_comments_only(bench, tmp_path, monkeypatch):
    src = os.path.join(ROOT, "paper_2307_14774_gb300", "csrc", "spc5_spmv.cu")
    text = open(src).read()
    fake = tmp_path / "paper_2307_14774_gb300" / "csrc"
    fake.mkdir(parents=True)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (fake / "spc5_spmv.cu").write_text(text)
    h0 = bench.kernel_source_hash()
    (fake / "spc5_spmv.cu").write_text("// a new comment\n" + text.replace("\n\n", "\n\n\n", 3))
    assert bench.kernel_source_hash() == h0
    (fake / "spc5_spmv.cu").write_text(text.replace("kVRound = 256", "kVRound = 128", 1))
    assert bench.kernel_source_hash() != h0


def test_committed_dram_table_parses(bench, monkeypatch):
    """profiles/spc5_spmv_dram.txt holds one DRAM figure per benchmark case;
    bench.py uses it only while its source hash is the kernels' (else the
    roofline's traffic is null)."""
    path = os.path.join(ROOT, "profiles", "spc5_spmv_dram.txt")
    stored = [ln.split(":", 1)[1].strip() for ln in open(path) if ln.startswith("source_sha256:")]
    assert len(stored) == 1
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: stored[0])
    table = bench.ncu_traffic()
    assert set(table) == {(m, f"{r}x{c}") for m in bench.MATRICES for r, c in bench.BETAS}
    assert all(v > 1e8 for v in table.values())
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.ncu_traffic() is None
