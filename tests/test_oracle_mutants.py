"""Planted mistakes: the oracle's pins must catch a plausible error anywhere in
it.  Each case copies oracle/hc_oracle.c to a temporary directory, plants one
mistake by text substitution (on the CPU only), compiles the copy, and checks
that a pin fails: the exhaustive brute-force comparison with the naive matcher
for mistakes that change the result set, the hand-worked hash values of Eq. 3
for mistakes that only change the hash.
"""
import ctypes
import os
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "hc_oracle.c")

# (name, original text, planted text) -- each must occur exactly once
RESULT_MUTANTS = [
    # the output position exactly as printed in the paper (one before the
    # window start): verified and reported there
    ("paper_literal_position", "    if (h == hv && memcmp(t + wstart, x, (size_t)m) == 0) *hit = 1;",
     "    if (h == hv && memcmp(t + wstart - 1, x, (size_t)m) == 0) *hit = 1;"),
    # shift one too far on a first-test miss
    ("shift_too_far", "        if (F[h] == 0) {\n            end += m - q + 1;",
     "        if (F[h] == 0) {\n            end += m - q + 2;"),
    # link stored in the left q-gram's word instead of the right one's (Eq. 1)
    ("link_transposed", "F[right] |= or_link_hash(left);", "F[left] |= or_link_hash(right);"),
    # marking phase (Eq. 2) dropped
    ("no_marking", "if (F[u] == 0) F[u] = 1;", "(void)u;"),
    # one chain too few
    ("chain_count", "long first_end = m - ((m - q + 1 < q) ? (m - q + 1) : q);",
     "long first_end = m - ((m - q < q) ? (m - q) : q);"),
    # the back-walk stops one q-gram early but the window counts as read in
    # full: the walk is too short AND H_v compares a different q-gram
    ("walk_bound", "while (last - 2 * q + 1 >= wstart) {",
     "while (last - 3 * q + 1 >= wstart) {"),
]

HASH_MUTANTS = [
    # characters read forwards: weights reversed (Eq. 3)
    ("hash_reversed", "for (long i = p; i >= p - q + 1; i--) v = (v << s) + (uint32_t)x[i];",
     "for (long i = p - q + 1; i <= p; i++) v = (v << s) + (uint32_t)x[i];"),
    # shift s taken as ceil(alpha / q) (Eq. 4)
    ("shift_ceil", "int s = alpha / q;                   /* Eq. 4 */",
     "int s = (alpha + q - 1) / q;"),
]


def _plant(td, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique/present: {old[:50]!r}"
    path = os.path.join(td, "hc_oracle_mut.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    return path


@pytest.mark.parametrize("name,old,new", RESULT_MUTANTS, ids=[m[0] for m in RESULT_MUTANTS])
def test_result_mutant_is_caught(name, old, new):
    with tempfile.TemporaryDirectory() as td:
        path = _plant(td, old, new)
        exe = os.path.join(td, "bf")
        subprocess.run(["gcc", "-O2", "-std=c99", "-o", exe,
                        os.path.join(ROOT, "tests", "brute_force.c"), path], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    if out.returncode != 0:
        return  # crashed (e.g. read before the text): caught
    r = {k: int(v) for k, v in (t.split("=") for t in out.stdout.split())}
    assert r["hc_mismatch"] > 0, name


@pytest.mark.parametrize("name,old,new", HASH_MUTANTS, ids=[m[0] for m in HASH_MUTANTS])
def test_hash_mutant_is_caught(name, old, new, golden_dir):
    with tempfile.TemporaryDirectory() as td:
        path = _plant(td, old, new)
        so = os.path.join(td, "libmut.so")
        subprocess.run(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", so, path],
                       check=True)
        lib = ctypes.CDLL(so)
        lib.or_preprocess.restype = ctypes.c_int
        mismatches = 0
        with open(os.path.join(golden_dir, "hash_eq3.txt")) as f:
            rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
        for hexbytes, q, alpha, want in rows:
            u = bytes.fromhex(hexbytes)
            q, alpha, want = int(q), int(alpha), int(want)
            # H_v of the pattern u itself is h(u) when m = q (a single q-gram)
            F = (ctypes.c_uint32 * (1 << alpha))()
            s, mask, hv = ctypes.c_int(), ctypes.c_uint32(), ctypes.c_uint32()
            buf = (ctypes.c_uint8 * len(u)).from_buffer_copy(u)
            rc = lib.or_preprocess(buf, ctypes.c_long(len(u)), q, alpha, F,
                                   ctypes.byref(s), ctypes.byref(mask), ctypes.byref(hv),
                                   None, ctypes.c_long(0), None, None)
            assert rc == 0
            mismatches += hv.value != want
        assert mismatches > 0, name
