"""Plant plausible mistakes in copies of the oracle and check that a pin catches each.

Each mutant is a textual edit of oracle/slab_oracle.c compiled into a temporary
library. The real oracle is never modified. A mutant that every pin accepts
would mean the pins leave that part of the oracle unchecked.
"""
import os
import subprocess
import tempfile

import pytest

from oracle.oracle import load_oracle
from tests.oracle_pins import ALL_PINS

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "slab_oracle.c")

MUTANTS = {
    "hash_drops_b": ("(uint64_t)a * (uint64_t)key + (uint64_t)b", "(uint64_t)a * (uint64_t)key"),
    "hash_swaps_a_b": ("(uint64_t)a * (uint64_t)key + (uint64_t)b",
                       "(uint64_t)b * (uint64_t)key + (uint64_t)a"),
    "hash_wrong_prime": ("#define OR_PRIME 4294967291ull", "#define OR_PRIME 4294967279ull"),
    "hash_skips_mod_p": ("(x % OR_PRIME) % num_buckets", "x % num_buckets"),
    "tombstone_matches": ("if (bk->s[s].live == OR_LIVE && bk->s[s].key == key)", "if (bk->s[s].key == key)"),
    "multiset_insert_lines_to_tail": (
        "while (s < bk->len && bk->s[s].live != OR_HOLE) s++;\n    if (lines) *lines += (uint64_t)s / t->M + 1;",
        "while (s < bk->len && bk->s[s].live != OR_HOLE) s++;\n    if (lines) *lines += (uint64_t)bk->len / t->M + 1;"),
    "multiset_insert_appends": ("while (s < bk->len && bk->s[s].live != OR_HOLE) s++;", "s = bk->len;"),
    "multiset_delete_tombstones": ("bk->s[s].live = t->multiset ? OR_HOLE : OR_TOMB;", "bk->s[s].live = OR_TOMB;"),
    "delete_all_first_only": ("                    kill(t, bk, s);\n                    c++;\n",
                              "                    kill(t, bk, s);\n                    c++;\n                    break;\n"),
    "search_all_counts_twice": ("values[i * cap + c] = t->key_only ? 0u : bk->s[s].value;\n                c++;",
                                "values[i * cap + c] = t->key_only ? 0u : bk->s[s].value;\n                c += 2;"),
    "flush_keeps_tombstones": ("if (bk->s[s].live == OR_LIVE) bk->s[w++] = bk->s[s];",
                               "if (bk->s[s].live != OR_HOLE) bk->s[w++] = bk->s[s];"),
    "flush_reverses_order": ("if (bk->s[s].live == OR_LIVE) bk->s[w++] = bk->s[s];",
                             "if (bk->s[s].live == OR_LIVE) { or_slot x = bk->s[s]; for (uint32_t q = w++; q > 0; q--) bk->s[q] = bk->s[q - 1]; bk->s[0] = x; }"),
    "slab_count_off_by_one": ("(len + t->M - 1) / t->M", "len / t->M + 1"),
    "wrong_pairs_per_slab": ("t->M = key_only ? W - 2u : (W - 2u) / 2u;", "t->M = key_only ? W - 2u : W / 2u;"),
    "slab_width_ignored": ("const uint32_t W = slab_bytes / 4u;", "const uint32_t W = 32u; (void)slab_bytes;"),
    "aux_word_holds_a_key": ("t->M = key_only ? W - 2u : (W - 2u) / 2u;", "t->M = key_only ? W - 1u : (W - 2u) / 2u;"),
    "search_lines_off_by_one": (
        "*value = t->key_only ? 0 : bk->s[s].value;\n        if (lines) *lines += (uint64_t)s / t->M + 1;",
        "*value = t->key_only ? 0 : bk->s[s].value;\n        if (lines) *lines += (uint64_t)s / t->M;"),
    "delete_result_always_one": ("r = (uint32_t)f;", "r = 1u;"),
    "insert_result_inverted": ("r = f ? 0u : 1u;", "r = f ? 1u : 0u;"),
    "replace_keeps_old_value": ("bk->s[s].value = value;", "(void)value;"),
    "utilization_drops_pointer": ("double y = 8.0;", "double y = 0.0;"),
    "bitmap_word_index": ("uint64_t w = block * 32 + unit / 32;", "uint64_t w = block * 32 + unit % 32;"),
    "address_field_width": ("uint32_t blk = (a >> 10) & 0x3FFFu;", "uint32_t blk = (a >> 12) & 0x3FFFu;"),
    "learned_root_target": ("add_point(&sx, &sy, &sxx, &sxy, x[i], i * 1024);", "add_point(&sx, &sy, &sxx, &sxy, x[i], i * 1000);"),
    "learned_unsorted_sample": ("qsort(x, m, sizeof(uint32_t), cmp_u32);", "(void)cmp_u32;"),
    "learned_empty_leaf_start": ("        below += cnt;\n", ""),
    "learned_intercept_sign": ("double u = u128_to_double(sy) - t;", "double u = u128_to_double(sy) + t;"),
    "learned_leaf_lookup": ("return linear_piece(model[2 + 2 * leaf], model[3 + 2 * leaf], x, num_buckets);",
                            "return linear_piece(model[3 + 2 * leaf], model[2 + 2 * leaf], x, num_buckets);"),
}


@pytest.fixture(scope="module")
def source():
    with open(SRC) as f:
        return f.read()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, source, tmp_path):
    old, new = MUTANTS[name]
    assert source.count(old) >= 1, f"mutation site for {name} not found"
    src = tmp_path / f"{name}.c"
    src.write_text(source.replace(old, new, 1))
    lib_path = str(tmp_path / f"lib{name}.so")
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC", "-o", lib_path,
                           str(src)])
    lib = load_oracle(lib_path)
    caught = []
    for pin in ALL_PINS:
        try:
            pin(lib)
        except AssertionError:
            caught.append(pin.__name__)
            break
    assert caught, f"no pin detects mutant {name}"


def test_real_oracle_passes_every_pin():
    lib = load_oracle()
    for pin in ALL_PINS:
        pin(lib)
