"""The oracle's pins have teeth: plausible mistakes are planted in a copy of
the oracle's C source (on the CPU only), each copy is compiled to its own
library under oracle/_build/mutants, and a fixed set of the pins of
test_oracle_pins.py, run against that library, must fail for every one of
them.  The mistakes are the kinds a restatement of the paper could make: a
wrong sign in the 2x2 rotation or in the rotation's application, a
transposed V-hat in the block-row update (Algorithm 2), a dropped term in
the block-column update, a wrong index in the round-robin table, a dropped
row in the Gram block (Sec. 6), a diagonal that stops carrying its low
word between rotations (the single-word diagonal that loses the energy of
late rotations), singular values sorted the wrong way, an off-norm that
counts the diagonal (Sec. 2.1, eq. (Omega_A)), and Algorithm 3's groups
shifted by one label."""
from __future__ import annotations

import os
import subprocess

import pytest

import oracle
import oracle.build as obuild

import test_oracle_pins as pins

MUTANTS = {
    "rotation_sign": (
        "tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + r);",
        "tt = (zeta >= 0.0 ? -1.0 : 1.0) / (fabs(zeta) + r);"),
    "rutishauser_sign": (
        "*y = b + s * (a - tau * b);",
        "*y = b - s * (a - tau * b);"),
    "row_update_transposed": (
        "for (int ii = 0; ii < k; ii++) s += AT(V, k, ii, jj) * x[ii];",
        "for (int ii = 0; ii < k; ii++) s += AT(V, k, jj, ii) * x[ii];"),
    "column_update_dropped_term": (
        "for (int ii = 0; ii < k; ii++) s += x[ii] * AT(V, k, ii, jj);",
        "for (int ii = 1; ii < k; ii++) s += x[ii] * AT(V, k, ii, jj);"),
    "round_robin_index": (
        "int bb = (pb == 0) ? 0 : 1 + ((pb - 1 + s) % (N - 1));",
        "int bb = (pb == 0) ? 0 : 1 + ((pb + s) % (N - 1));"),
    "gram_row_dropped": (
        "for (int r = 0; r < m; r++) s += AT(G, ldg, r, gi) * AT(G, ldg, r, gj);",
        "for (int r = 1; r < m; r++) s += AT(G, ldg, r, gi) * AT(G, ldg, r, gj);"),
    "svd_sorted_ascending": (
        "    stable_argsort(n, sg, idx, 0);",
        "    stable_argsort(n, sg, idx, 1);"),
    "off_norm_counts_the_diagonal": (
        "            if (i != j) s += AT(A, lda, i, j) * AT(A, lda, i, j);",
        "            s += AT(A, lda, i, j) * AT(A, lda, i, j);"),
    "anti_diagonal_group_shifted": (
        "                if ((I + J) % N == K) {",
        "                if ((I + J + 1) % N == K) {"),
    "diagonal_low_word_not_carried": (
        "err += *lo + dl;",
        "err += dl;"),
}

# the pins run against every mutant (each is cheap); at least one must fail
PINS = [
    (pins.test_rotation_matches_2x2_closed_form, ()),
    (pins.test_single_rotation_drops_off2_by_2apq2, (0,)),
    (pins.test_known_spectrum_blocked, (8, oracle.ORDER_ROUND_ROBIN, "uniform")),
    (pins.test_trace_and_frobenius_invariance_through_steps, ()),
    (pins.test_step_pivot_blocks_hold_dhat_and_match_explicit_product, (1,)),
    (pins.test_round_robin_covers_every_pair_once, (8,)),
    (pins.test_known_singular_values, (False, 4)),
    (pins.test_pivot_solve_preserves_energy_without_bias, ()),
    (pins.test_pivot_eigenvectors_keep_unit_length, ()),
    (pins.test_algorithm3_matches_printed_label_matrix, ()),
]


def _build_mutant(name: str) -> str:
    src = open(obuild.SRC).read()
    before, after = MUTANTS[name]
    assert src.count(before) == 1, f"mutation site of {name} not found exactly once"
    out_dir = os.path.join(obuild.OUT_DIR, "mutants")
    os.makedirs(out_dir, exist_ok=True)
    csrc = os.path.join(out_dir, f"{name}.c")
    lib = os.path.join(out_dir, f"lib{name}.so")
    with open(csrc, "w") as f:
        f.write(src.replace(before, after))
    subprocess.run(["gcc"] + obuild.CFLAGS + ["-o", lib, csrc, "-lm"], check=True)
    return lib


def _failing_pins():
    failed = []
    for fn, args in PINS:
        try:
            fn(*args)
        except (AssertionError, ValueError, ArithmeticError):
            failed.append(fn.__name__)
    return failed


def test_pins_pass_on_the_oracle_itself():
    assert _failing_pins() == []


@pytest.mark.filterwarnings("ignore::RuntimeWarning")   # a mutant's overflowing iterates
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_the_planted_mistake(name, monkeypatch):
    lib = _build_mutant(name)
    monkeypatch.setattr(oracle, "_LIB", None)
    monkeypatch.setattr(oracle._build, "build", lambda force=False: lib)
    failed = _failing_pins()
    assert failed, f"no pin catches the mutant {name}"
