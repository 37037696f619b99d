"""The oracle's pins must reject plausible mistakes (no GPU).

Each mutant is a copy of ``oracle/onesweep_oracle.c`` with one deliberate
error, compiled into a temporary directory and checked by ``oracle_pins.py``
in a child process. Every mutant must fail at least one pin; the real oracle
must fail none.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "onesweep_oracle.c")
PINS = os.path.join(ROOT, "tests", "oracle_pins.py")

MUTANTS = {
    "inclusive_instead_of_exclusive": ("out[i] = running;\n        running += v;",
                                       "running += v;\n        out[i] = running;"),
    "msd_place_order": ("place_bits(begin_bit, end_bit, radix_bits, place, &shift, &width);\n        binning_pass",
                        "place_bits(begin_bit, end_bit, radix_bits, p - 1 - place, &shift, &width);\n        binning_pass"),
    "value_does_not_follow_key": ("if (vin) vout[dst] = vin[i];", "if (vin) vout[i] = vin[i];"),
    "digit_mask_off_by_one": ("uint64_t mask = (width >= 64) ? ~0ULL : ((1ULL << width) - 1ULL);",
                              "uint64_t mask = (width >= 64) ? ~0ULL : ((1ULL << width) - 2ULL);"),
    "f32_negatives_not_inverted": ("(uint32_t)~b : (b | 0x80000000u)", "(b ^ 0x80000000u) : (b | 0x80000000u)"),
    "f32_wrong_inverse": ("(v & 0x7FFFFFFFu) : (uint32_t)~v", "(v & 0x7FFFFFFFu) : (v ^ 0x80000000u)"),
    "f64_transform_missing": ("return (bits & sign) ? ~bits : (bits | sign);", "return bits;"),
    "last_place_not_narrowed": ("*width = w < radix_bits ? w : radix_bits;", "*width = radix_bits;"),
    "histogram_skips_transform": ("hist[place * r + sort_digit(u, shift, width, descending)] += 1;",
                                  "hist[place * r + sort_digit(load_key(key_type, keys, i), shift, width, "
                                  "descending)] += 1;"),
    "tile_index_wrong": ("counts[(i / tile) * r", "counts[(i / (tile + 1)) * r"),
    "places_start_at_zero": ("*shift = begin_bit + place * radix_bits;", "*shift = place * radix_bits;"),
    "signed_keys_not_flipped": ("if (key_type == ORC_I32) return (uint32_t)bits ^ 0x80000000u;",
                                "if (key_type == ORC_I32) return (uint32_t)bits;"),
    "descending_ignored": ("return descending ? ((1ULL << width) - 1ULL) - d : d;", "return d;"),
    "descending_complement_off_by_one": ("return descending ? ((1ULL << width) - 1ULL) - d : d;",
                                         "return descending ? ((1ULL << width) - 1ULL) - d - (d == 0 ? 0 : 1) : d;"),
    "descending_histogram_plain": ("hist[place * r + sort_digit(u, shift, width, descending)] += 1;",
                                   "hist[place * r + digit_of(u, shift, width)] += 1;"),
}


def _run_pins(lib):
    out = subprocess.run([sys.executable, PINS, lib], capture_output=True, text=True, timeout=300)
    if out.returncode != 0:
        return ["<crashed>"]
    return json.loads(out.stdout.strip().splitlines()[-1])


def test_real_oracle_passes_all_pins(tmp_path):
    lib = tmp_path / "liboracle_real.so"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", SRC, "-o", str(lib)])
    assert _run_pins(str(lib)) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mutant = tmp_path / f"{name}.c"
    mutant.write_text(src.replace(old, new))
    lib = tmp_path / f"lib{name}.so"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", str(mutant), "-o", str(lib)])
    assert _run_pins(str(lib)) != [], f"no pin rejects the {name} mutant"
