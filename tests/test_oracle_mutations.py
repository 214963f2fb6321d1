"""The oracle's pins are strong enough to catch plausible mistakes.

Each case copies the oracle source, plants one mistake of the kind a reader
could make when writing it from the paper (a flipped tie rule, a wrong
equality-bucket index, a dropped term, a reversed comparison, a wrong key
map), compiles the copy, and runs the oracle pin suite against it in a child
process.  The suite must fail for every mutant.  Nothing here touches the GPU.
"""
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ips4o_oracle.c")

MUTANTS = {
    # Section 3 tie rule s_i <= e < s_{i+1} turned into s_i < e <= s_{i+1}
    "tie_rule": ("if (key_less(e, spl[mid])) hi = mid; else lo = mid + 1;",
                 "if (!key_less(spl[mid], e)) hi = mid; else lo = mid + 1;"),
    # Section 4.4: keys equal to s_i sent to the range bucket instead
    "eq_bucket_index": ("return 2 * i - 1;", "return 2 * i;"),
    # duplicate splitters not removed (Section 4.7)
    "no_dedup": ("if (m > 0 && key_eq(c, spl[m - 1])) { dup = 1; continue; }",
                 "if (0) { dup = 1; continue; }"),
    # inclusive instead of exclusive prefix sum for bucket starts
    "prefix_sum": ("{ L->bounds[b] = sum; sum += cnt[b]; }",
                   "{ sum += cnt[b]; L->bounds[b] = sum - cnt[b] + (b > 0); }"),
    # base case sorts descending
    "insertion_cmp": ("while (j > 0 && key_less(ki, key_of(a + (j - 1) * s, kt)))",
                      "while (j > 0 && key_less(key_of(a + (j - 1) * s, kt), ki))"),
    # float map forgets to invert negative numbers
    "f64_map": ("k.hi = (v >> 63) ? ~v : (v | 0x8000000000000000ULL);",
                "k.hi = v ^ 0x8000000000000000ULL;"),
    # record key bytes 8 and 9 swapped
    "rec100_lo": ("k.lo = ((uint64_t)e[8] << 8) | e[9];",
                  "k.lo = ((uint64_t)e[9] << 8) | e[8];"),
    # splitters taken one place off the equal spacing of Section 3
    "splitter_spacing": ("okey c = sample[(size_t)j * alpha - 1];",
                         "okey c = sample[(size_t)j * alpha - (j < k - 1 ? 0 : 1)];"),
    # the third key word of a quartet ignored in comparisons (Section 5)
    "quartet_third_word": ("return a.hi < b.hi || (a.hi == b.hi && (a.lo < b.lo || (a.lo == b.lo && a.lo2 < b.lo2)));",
                           "return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);"),
    # range buckets skipped instead of equality buckets during recursion
    "recurse_skip": ("if (L.eq && (b % 2 == 1)) continue;",
                     "if (L.eq && (b % 2 == 0)) continue;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mut_src = tmp_path / "mutant.c"
    mut_src.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O1", "-shared", "-fPIC", "-std=c11", str(mut_src), "-o", str(lib), "-lm"],
                   check=True)
    env = dict(os.environ, IPS4O_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the oracle pins:\n{r.stdout[-2000:]}"


def test_unmutated_source_passes():
    # the same harness with the real oracle passes (guards against a harness
    # that fails for every library)
    lib = oracle.build()
    env = dict(os.environ, IPS4O_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle.py"), "-k", "partition or f64 or rec100"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:]
