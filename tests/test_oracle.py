"""CPU-only tests: the oracle against its pins, and the pins against mutants.

A pin that cannot tell a wrong oracle from a right one pins nothing, so the
second half compiles mutated copies of the oracle's C source (each a
plausible mistake: a dropped pass, a digit taken from the wrong byte, an
unstable scatter, a signed reading of the keys, a value that does not travel
with its key, a histogram that misses a digit) and checks that at least one
pin rejects every mutant.  The mutants run here, on the CPU, only.
"""
from __future__ import annotations

import os
import subprocess

import pytest

import oracle
from tests import oracle_pins


@pytest.mark.parametrize("pin", oracle_pins.ALL_PINS, ids=lambda f: f.__name__)
def test_oracle_pin(pin):
    pin()


def test_paper_byte_model_golden():
    """Sec. 5: 64 Mi pairs x 8 B x 4 passes = 2048 MiB written per sort."""
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_byte_model.txt")
    vals = {}
    for line in open(path):
        line = line.split("#", 1)[0].strip()
        if line:
            key, val = line.split("=")
            vals[key.strip()] = int(val)
    n = vals["items"]
    written = n * vals["bytes_per_item"] * vals["passes"]
    assert written == vals["ideal_written_mib"] * 2**20
    # The measured figure is a little lower (final pass not fully streamed).
    assert vals["measured_written_mib"] <= vals["ideal_written_mib"]
    from paper_1008_2849_gb300 import roofline
    assert roofline.scatter_bytes_per_item(with_values=True) * vals["passes"] * n \
        == 2 * written  # reads equal writes in our accounting


MUTANTS = {
    "dropped_pass": ("for (unsigned p = 0; p < PASSES; ++p) {\n        oracle_counting_pass",
                     "for (unsigned p = 0; p < PASSES - 2; ++p) {\n        oracle_counting_pass"),
    "wrong_byte": ("return (key >> (RADIX_BITS * p)) & (RADIX - 1u);",
                   "return (key >> (RADIX_BITS * (p ^ 1u))) & (RADIX - 1u);"),
    "msd_first": ("return (key >> (RADIX_BITS * p)) & (RADIX - 1u);",
                  "return (key >> (RADIX_BITS * (3u - p))) & (RADIX - 1u);"),
    "signed_top_byte": ("return (key >> (RADIX_BITS * p)) & (RADIX - 1u);",
                        "return ((key >> (RADIX_BITS * p)) & (RADIX - 1u)) ^ (p == 3u ? 0x80u : 0u);"),
    "unstable_scatter": ("    for (size_t i = 0; i < n; ++i) {\n        uint32_t b = digit_of(keys_src[i], p);\n        uint64_t slot = next[b];\n        next[b] = slot + 1;",
                         "    for (size_t r = 0; r < n; ++r) {\n        size_t i = n - 1 - r;\n        uint32_t b = digit_of(keys_src[i], p);\n        uint64_t slot = next[b];\n        next[b] = slot + 1;"),
    "value_left_behind": ("if (vals_src) vals_dst[slot] = vals_src[i];",
                          "if (vals_src) vals_dst[slot] = vals_src[slot];"),
    "histogram_skips_top_digit": ("        for (unsigned p = 0; p < PASSES; ++p)\n            hist[p * RADIX + digit_of(keys[i], p)] += 1;",
                                  "        for (unsigned p = 0; p < PASSES - 1; ++p)\n            hist[p * RADIX + digit_of(keys[i], p)] += 1;"),
    "inclusive_prefix": ("            first[p * RADIX + b] = run;\n            run += hist[p * RADIX + b];",
                         "            run += hist[p * RADIX + b];\n            first[p * RADIX + b] = run;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(name, tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "rs_oracle.c")).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, "mutation anchor not found: %s" % name
    mutated = tmp_path / ("%s.c" % name)
    mutated.write_text(src.replace(old, new))
    so = tmp_path / ("lib%s.so" % name)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                           "-o", str(so), str(mutated)])
    lib = oracle._bind(str(so))
    failures = []
    for pin in oracle_pins.ALL_PINS:
        try:
            pin(lib)
        except AssertionError:
            failures.append(pin.__name__)
    assert failures, "no pin rejects mutant %s" % name


@pytest.mark.parametrize("pin", oracle_pins.TYPED_PINS, ids=lambda f: f.__name__)
def test_typed_oracle_pin(pin):
    pin()


TYPED_MUTANTS = {
    "float_negatives_ascending": ("    return ma > mb;                /* both negative */",
                                  "    return ma < mb;                /* both negative */"),
    "signed_read_as_unsigned": ("    if (key_type == 1) return (int32_t)a < (int32_t)b;",
                                "    if (key_type == 1) return a < b;"),
    "unstable_merge": ("        if (typed_less(keys[idx[j]], keys[idx[i]], key_type))",
                       "        if (!typed_less(keys[idx[i]], keys[idx[j]], key_type))"),
    "zeros_equal": ("    if (sa != sb) return sa > sb;  /* negative sign first */",
                    "    if (sa != sb) return (ma | mb) != 0 && sa > sb;"),
    "nan_payload_ignored": ("    const uint32_t ma = a & 0x7fffffffu, mb = b & 0x7fffffffu;",
                            "    const uint32_t ma = (a & 0x7fffffffu) > 0x7f800000u ? 0x7f800001u : (a & 0x7fffffffu),\n"
                            "                   mb = (b & 0x7fffffffu) > 0x7f800000u ? 0x7f800001u : (b & 0x7fffffffu);"),
}


@pytest.mark.parametrize("name", sorted(TYPED_MUTANTS))
def test_typed_pins_reject_mutant(name, tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "rs_oracle.c")).read()
    old, new = TYPED_MUTANTS[name]
    assert src.count(old) == 1, "mutation anchor not found: %s" % name
    mutated = tmp_path / ("%s.c" % name)
    mutated.write_text(src.replace(old, new))
    so = tmp_path / ("lib%s.so" % name)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                           "-o", str(so), str(mutated)])
    lib = oracle._bind(str(so))
    failures = []
    for pin in oracle_pins.TYPED_PINS:
        try:
            pin(lib)
        except AssertionError:
            failures.append(pin.__name__)
    assert failures, "no pin rejects mutant %s" % name


@pytest.mark.parametrize("pin", oracle_pins.KEY64_PINS, ids=lambda f: f.__name__)
def test_key64_oracle_pin(pin):
    pin()


KEY64_MUTANTS = {
    "only_four_passes": ("    for (unsigned p = 0; p < PASSES64; ++p) {\n        counting_pass64",
                         "    for (unsigned p = 0; p < PASSES; ++p) {\n        counting_pass64"),
    "digit_from_low_word": ("    return (uint32_t)((key >> (RADIX_BITS * p)) & (RADIX - 1u));",
                            "    return (uint32_t)(((uint32_t)key >> (RADIX_BITS * (p & 3u))) & (RADIX - 1u));"),
    "value_left_behind64": ("        if (vals_src != NULL) vals_dst[slot] = vals_src[i];",
                            "        if (vals_src != NULL) vals_dst[i] = vals_src[i];"),
}


@pytest.mark.parametrize("name", sorted(KEY64_MUTANTS))
def test_key64_pins_reject_mutant(name, tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "rs_oracle.c")).read()
    old, new = KEY64_MUTANTS[name]
    assert src.count(old) == 1, "mutation anchor not found: %s" % name
    mutated = tmp_path / ("%s.c" % name)
    mutated.write_text(src.replace(old, new))
    so = tmp_path / ("lib%s.so" % name)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                           "-o", str(so), str(mutated)])
    lib = oracle._bind(str(so))
    failures = []
    for pin in oracle_pins.KEY64_PINS:
        try:
            pin(lib)
        except AssertionError:
            failures.append(pin.__name__)
    assert failures, "no pin rejects mutant %s" % name


@pytest.mark.parametrize("pin", oracle_pins.KV_PINS, ids=lambda f: f.__name__)
def test_kv_oracle_pin(pin):
    pin()


KV_MUTANTS = {
    "i64_compared_unsigned": ("    if (key_type == 4) return (int64_t)x < (int64_t)y;",
                              "    if (key_type == 4) return x < y;"),
    "f64_negatives_not_reversed": ("    return mx > my;                /* both negative */",
                                   "    return mx < my;                /* both negative */"),
    "value_half_carried": ("(const unsigned char*)vals_in + vb * idx[i],\n                   vb);",
                           "(const unsigned char*)vals_in + vb * idx[i],\n                   4);"),
    "unstable_merge": ("        if (kv_less(keys, idx[j], idx[i], key_type))",
                       "        if (!kv_less(keys, idx[i], idx[j], key_type))"),
    "f64_read_as_i64": ("    if (key_type == 3) return x < y;\n    if (key_type == 4)",
                        "    if (key_type == 3) return x < y;\n    if (key_type >= 4)"),
}


@pytest.mark.parametrize("name", sorted(KV_MUTANTS))
def test_kv_pins_reject_mutant(name, tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "rs_oracle.c")).read()
    old, new = KV_MUTANTS[name]
    assert src.count(old) == 1, "mutation anchor not found: %s" % name
    mutated = tmp_path / ("%s.c" % name)
    mutated.write_text(src.replace(old, new))
    so = tmp_path / ("lib%s.so" % name)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                           "-o", str(so), str(mutated)])
    lib = oracle._bind(str(so))
    failures = []
    for pin in oracle_pins.KV_PINS:
        try:
            pin(lib)
        except AssertionError:
            failures.append(pin.__name__)
    assert failures, "no pin rejects mutant %s" % name
