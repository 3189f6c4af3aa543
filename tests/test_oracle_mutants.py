"""The oracle's pins must catch plausible mistakes.

Each case compiles a copy of the oracle source with one deliberate mistake
(a dropped term, a wrong index, a wrong order, ...) into a temporary library
on the CPU and runs a few of the pin checks against it; at least one of them
has to fail. This shows the pins constrain every step, not just a few.
"""
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from paper_2208_09985_gb300 import synth
from tests import _brute as brute

SRC = os.path.join(os.path.dirname(oracle.__file__), "genasm_oracle.c")

MUTANTS = {
    "dc_drop_deletion_term": ("bv_and(bv_and(I, D), bv_and(S, M))", "bv_and(I, bv_and(S, M))"),
    "dc_insertion_wrong_column": ("bv I = bv_shl1(t->R[AT(t, i, d - 1)]);",
                                  "bv I = bv_shl1(t->R[AT(t, i + 1, d - 1)]);"),
    "dc_match_wrong_row": ("bv M = bv_or(bv_shl1(t->R[AT(t, i + 1, d)]), cur);",
                           "bv M = bv_or(bv_shl1(t->R[AT(t, i + 1, d - 1)]), cur);"),
    "init_off_by_one": ("bv_ones_shl(m, d);\n    /* the insertion", "bv_ones_shl(m, d + 1);\n    /* the insertion"),
    "pattern_mask_inverted": ("if (pattern[j] != x) bv_setbit", "if (pattern[j] == x) bv_setbit"),
    "tb_substitution_bit": ("bv_bit(&t->ED[AT(t, i, d)], j + 1) == 0) {\n            cigar_push(out, ORC_OP_X);",
                            "bv_bit(&t->ED[AT(t, i, d)], j) == 0) {\n            cigar_push(out, ORC_OP_X);"),
    "tb_stop_one_late": ("while (j < t->m && i < limit && j < limit)", "while (j < t->m && i <= limit && j < limit)"),
    "tb_order_I_before_S": (
        "} else if (d > 0 && i < t->n && bv_bit(&t->ED[AT(t, i, d)], j + 1) == 0) {\n            cigar_push(out, ORC_OP_X);\n            i += 1;\n            j += 1;\n            d -= 1;\n        } else if (d > 0 && bv_bit(&t->EI[AT(t, i, d)], j) == 0) {\n            cigar_push(out, ORC_OP_I);\n            j += 1;\n            d -= 1;",
        "} else if (d > 0 && bv_bit(&t->EI[AT(t, i, d)], j) == 0) {\n            cigar_push(out, ORC_OP_I);\n            j += 1;\n            d -= 1;\n        } else if (d > 0 && i < t->n && bv_bit(&t->ED[AT(t, i, d)], j + 1) == 0) {\n            cigar_push(out, ORC_OP_X);\n            i += 1;\n            j += 1;\n            d -= 1;"),
    "window_advance_ignores_indels": ("        ti += ci;\n        pj += cj;", "        ti += cj;\n        pj += cj;"),
    "edit_distance_last_row": ("for (int d = 0; d <= t->k; ++d)\n        if (bv_bit(&t->R[AT(t, 0, d)], 0) == 0) return d;",
                               "for (int d = t->k; d >= 0; --d)\n        if (bv_bit(&t->R[AT(t, 0, d)], 0) == 0) return d;"),
    "multiword_shift_no_carry": ("r.w[0] = (a.w[0] << 1) | (a.w[1] >> 63);", "r.w[0] = (a.w[0] << 1);"),
}


def _pins_pass(lib) -> bool:
    """A compact run of the pin checks against the oracle bound to ``lib``; True if all hold."""
    saved = oracle._lib
    oracle._lib = lib
    try:
        rng = np.random.default_rng(2)
        for _ in range(300):
            n, m = int(rng.integers(0, 9)), int(rng.integers(0, 9))
            t = rng.integers(0, 4, n).astype(np.uint8)
            p = rng.integers(0, 4, m).astype(np.uint8)
            k = max(n, m)
            bits, d_opt = oracle.window_table(t, p, k)
            dist = brute.free_end_table(t, p)[:, :m]
            expect = (dist[:, None, :] > np.arange(k + 1)[None, :, None]).astype(np.uint8)
            if not np.array_equal(bits, expect):
                return False
        for n, m in ((100, 97), (128, 128)):
            t = rng.integers(0, 4, n).astype(np.uint8)
            p = t[:m].copy()
            p[::7] = (p[::7] + 1) % 4
            bits, _ = oracle.window_table(t, p, 128)
            dist = brute.free_end_table(t, p)[:, :m]
            if not np.array_equal(bits, (dist[:, None, :] > np.arange(129)[None, :, None]).astype(np.uint8)):
                return False
        for it in range(150):
            W = int(rng.choice([8, 16, 32]))
            O = int(rng.integers(0, W))
            b = synth.random_pairs(1, 3 * W, 3 * W, seed=500 + it)
            t, p = b.text(0), b.pattern(0)
            r = oracle.align_pair(t, p, W, O)
            if r["status"] != 0:
                return False
            if brute.check_cigar(t, p, r["cigar"], r["text_consumed"], r["edit_count"]):
                return False
            if len(p) <= W - O and len(t) <= W and r["edit_count"] != brute.free_end_distance(t, p):
                return False
        for tx, px, want in (("AAAC", "AAC", "2=1X"), ("ACGT", "AGT", "1=1D2="), ("AGTT", "ACGT", "1=1I2=")):
            r = oracle.align_pair(synth.encode(tx), synth.encode(px), 8, 0)
            if oracle.cigar_string(r["cigar"]) != want:
                return False
        r = oracle.align_pair(synth.encode("ACGT" * 40), synth.encode("ACGT" * 25), 16, 6)
        if r["d_opt"].shape[0] != 10:
            return False
        t = synth.encode("ACGT" * 40)
        q = np.concatenate([t[:2], t[3:]])[:100]
        r = oracle.align_pair(t, q, 16, 6)
        if r["d_opt"].shape[0] != 11 or oracle.cigar_string(r["cigar"]) != "2=1D98=":
            return False
        return True
    except Exception:
        return False
    finally:
        oracle._lib = saved


def _compile(src_text: str, tmp: str, name: str) -> str:
    c = os.path.join(tmp, name + ".c")
    so = os.path.join(tmp, name + ".so")
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-pthread", c, "-o", so])
    return so


def test_unmodified_oracle_passes():
    src = open(SRC).read()
    with tempfile.TemporaryDirectory() as tmp:
        assert _pins_pass(oracle.bind(_compile(src, tmp, "orig")))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    src = open(SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    with tempfile.TemporaryDirectory() as tmp:
        lib = oracle.bind(_compile(src.replace(old, new), tmp, name))
        assert not _pins_pass(lib), f"mutant {name} passed every pin"
