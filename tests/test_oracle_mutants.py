"""Planted mistakes: each mutant of the oracle's C source (a dropped term, a
wrong sign, a wrong index or bound, a transposed operand) is compiled on the
CPU and must fail at least one pin, while the unmodified source passes them
all.  This checks that the pins constrain every oracle function."""
from __future__ import annotations

import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import synth
from bruteforce import grid_convert, pack_word

SRC = os.path.join(os.path.dirname(oracle.__file__), "spc5_oracle.c")

# (name, original text, replacement): every original must occur in the source
MUTANTS = [
    ("csr_sign", "double term = vals[e] * x[colidx[e]];",
     "double term = -vals[e] * x[colidx[e]];"),
    ("csr_index", "double term = vals[e] * x[colidx[e]];", "double term = vals[e] * x[e % 3];"),
    ("csr_drop_comp", "y[i] = s + comp;", "y[i] = s;"),
    ("csr_skip_first", "for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {\n      double term",
     "for (int64_t e = rowptr[i] + 1; e < rowptr[i + 1]; ++e) {\n      double term"),
    ("conv_width", "colidx[ptr[q]] < s + c)", "colidx[ptr[q]] <= s + c)"),
    ("conv_max_start", "colidx[ptr[q]] < s)) s = colidx[ptr[q]];",
     "colidx[ptr[q]] > s)) s = colidx[ptr[q]];"),
    ("conv_bit_reversed", "mask |= 1ULL << (colidx[ptr[q]] - s);",
     "mask |= 1ULL << (c - 1 - (colidx[ptr[q]] - s));"),
    ("conv_row_index", "int64_t row = p * r + q;\n      ptr[q]",
     "int64_t row = p + q;\n      ptr[q]"),
    ("alg1_x_offset", "sum[idxRowBlock] += x[idxCol + k] * values[idxVal];",
     "sum[idxRowBlock] += x[idxCol + k + 1] * values[idxVal];"),
    ("alg1_row_sum", "sum[idxRowBlock] += x[idxCol + k] * values[idxVal];",
     "sum[0] += x[idxCol + k] * values[idxVal];"),
    ("alg1_value_lag", "            idxVal += 1;\n", "            idxVal += (k & 1) ? 1 : 0;\n"),
    ("tocsr_col", "colidx_out[next[row]] = (int32_t)(block_colidx[b] + k);",
     "colidx_out[next[row]] = (int32_t)(block_colidx[b] + c - 1 - k);"),
    ("pack_shift", "<< (q * c);", "<< (q * 8);"),
    ("check_unsorted", "colidx[e] <= colidx[e - 1]) return ORACLE_EUNSORTED;",
     "colidx[e] < colidx[e - 1]) return ORACLE_EUNSORTED;"),
    ("bf16_double_rounding", "bf16_from_f32_rne(round_to_odd_f32(in[i]))",
     "bf16_from_f32_rne((float)in[i])"),
    ("bf16_truncate", "b += 0x7FFFu + lsb;", "b += 0u * lsb;"),
    ("hybrid_scalar_row", "s_rowptr[p * r + qs + 1]++;", "s_rowptr[p * r + 1]++;"),
    ("hybrid_scalar_value", "s_vals[next[row]] = values[idxVal];",
     "s_vals[next[row]] = values[idxVal > 0 ? idxVal - 1 : 0];"),
    ("hybrid_value_skip", "        idxVal += 1;\n      } else {",
     "        idxVal += 2;\n      } else {"),
    ("hybrid_keep_mask_row", "masks_b[kept * r + q] = block_masks[b * r + q];",
     "masks_b[kept * r + q] = block_masks[b * r];"),
]


def _compile(text: str, path: str):
    src = path + ".c"
    with open(src, "w") as f:
        f.write(text)
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", src, "-o", path, "-lm"],
                   check=True, capture_output=True)


def _pins(O: oracle.Oracle) -> list[str]:
    """Run the pins against one compiled oracle; return the names that fail."""
    failed = []

    def pin(name, fn):
        try:
            if not fn():
                failed.append(name)
        except Exception:
            failed.append(name)

    small = [synth.bernoulli(13, 29, d, seed=i) for i, d in enumerate((0.1, 0.4, 0.9))]
    small.append(synth.bernoulli(33, 40, 0.3, seed=5))

    def dense_exact():
        for A in small:
            x = synth.vector_int(A.ncols, -4, 4, seed=1)
            y, s = O.csr_spmv(A, x)
            if not np.array_equal(y, A.todense() @ x):
                return False
        return True

    def fsum_close():
        A = synth.powerlaw(1500, seed=11)
        x = synth.vector_uniform(A.ncols, seed=7)
        y, scale = O.csr_spmv(A, x)
        for i in range(A.nrows):
            lo, hi = A.rowptr[i], A.rowptr[i + 1]
            ref = math.fsum(float(v) * float(x[j]) for v, j in zip(A.vals[lo:hi], A.colidx[lo:hi]))
            if abs(y[i] - ref) > 2 * np.finfo(float).eps * abs(ref) + 1e-30 * scale[i]:
                return False
        return True

    def grid(rc_list):
        def f():
            for A in small:
                for r, c in rc_list:
                    S = O.convert(A, r, c)
                    brp, cols, masks, values = grid_convert(A, r, c)
                    if (S.block_rowptr.tolist() != brp or S.block_colidx.tolist() != cols
                            or S.block_masks.tolist() != masks or S.values.tolist() != values):
                        return False
                    nbytes = (r * c + 7) // 8
                    expect = [[(pack_word(m, c) >> (8 * t)) & 0xFF for t in range(nbytes)]
                              for m in masks]
                    if S.packed_masks().tolist() != expect:
                        return False
            return True
        return f

    def alg1_exact():
        for A in small:
            x = synth.vector_int(A.ncols, -5, 5, seed=2)
            for r, c in ((1, 8), (4, 4), (8, 4)):
                if not np.array_equal(O.spc5_spmv(O.convert(A, r, c), x), A.todense() @ x):
                    return False
        return True

    def roundtrip():
        for A in small + [synth.stencil27(7, 6, 5)]:
            for r, c in ((2, 4), (4, 8)):
                rp, ci, v = O.to_csr(O.convert(A, r, c))
                if not (np.array_equal(rp, A.rowptr) and np.array_equal(ci, A.colidx)
                        and np.array_equal(v, A.vals)):
                    return False
        return True

    def rejects_duplicates():
        A = synth.bernoulli(6, 6, 0.6, seed=1)
        dup = A.colidx.copy()
        a = A.rowptr[int(np.argmax(np.diff(A.rowptr) >= 2))]
        dup[a + 1] = dup[a]
        return O.check_csr(6, 6, A.rowptr, dup) == 2

    def closed_form():
        A = synth.laplace2d(128, 128)
        return (O.convert(A, 1, 8).nblocks == 48896 and O.convert(A, 4, 8).nblocks == 12224)

    pin("dense_exact", dense_exact)
    pin("fsum_close", fsum_close)
    pin("grid_convert", grid([(1, 8), (2, 4), (4, 8), (3, 5)]))
    pin("alg1_exact", alg1_exact)
    pin("roundtrip", roundtrip)
    pin("rejects_duplicates", rejects_duplicates)
    def quantize_exact():
        from test_oracle_quantize import _cases, bf16_exact
        v = _cases()
        got = O.quantize(v, "bf16")
        if not np.array_equal(got, np.array([bf16_exact(float(d)) for d in v], np.uint16)):
            return False
        return np.array_equal(O.quantize(v, "f32").view(np.uint32),
                              v.astype(np.float32).view(np.uint32))

    def hybrid():
        from test_oracle_hybrid import _expected
        for A in small + [synth.stencil27(7, 6, 5)]:
            for r, c in ((1, 8), (2, 4), (4, 8), (3, 5)):
                S = O.convert(A, r, c)
                B, Sc = O.hybrid_split(S)
                keep, scalars, vals_keep = _expected(S)
                scalars.sort(key=lambda t: (t[0], t[1]))
                if not (np.array_equal(B.block_colidx, S.block_colidx[keep])
                        and np.array_equal(B.block_masks, S.block_masks[keep])
                        and np.array_equal(B.values, vals_keep)
                        and np.array_equal(Sc.colidx, [t[1] for t in scalars])
                        and np.array_equal(Sc.vals, [t[2] for t in scalars])
                        and np.array_equal(np.diff(Sc.rowptr), np.bincount(
                            [t[0] for t in scalars], minlength=A.nrows))):
                    return False
        return True

    pin("closed_form", closed_form)
    pin("quantize_exact", quantize_exact)
    pin("hybrid", hybrid)
    return failed


def _pins_in_child(path: str) -> list[str]:
    """Run the pins in a fresh interpreter: a mutant may corrupt memory, and
    a crash of the child counts as a failed pin."""
    code = ("import json, sys; sys.path[:0] = [%r, %r]; import test_oracle_mutants as m, oracle; "
            "print(json.dumps(m._pins(oracle.Oracle(%r))))"
            % (os.path.dirname(__file__), os.path.dirname(os.path.dirname(__file__)), path))
    proc = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                          timeout=600)
    if proc.returncode != 0:
        return ["child crashed"]
    return json.loads(proc.stdout.strip().splitlines()[-1])


def test_unmodified_oracle_passes_all_pins(tmp_path):
    path = str(tmp_path / "liboracle_orig.so")
    _compile(open(SRC).read(), path)
    assert _pins_in_child(path) == []


@pytest.mark.parametrize("name,orig,repl", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, name, orig, repl):
    text = open(SRC).read()
    assert orig in text, f"mutation site for {name} not found"
    path = str(tmp_path / f"liboracle_{name}.so")
    _compile(text.replace(orig, repl, 1), path)
    failed = _pins_in_child(path)
    assert failed, f"mutant {name} passed every pin"
