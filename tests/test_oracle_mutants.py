"""The pins are strong enough: plant plausible mistakes in a copy of the
oracle's C source (CPU only) and check that every one of them makes at least
one pin fail.  The real oracle is untouched.
"""
import json
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

import test_oracle_pins as pins
from oracle import oracle as O

# (name, original text, planted mistake); each original must occur exactly once.
MUTANTS = [
    ("extend uses open (score)", "E = max2(E - e, Hleft - o);                 /* E(i,j) */",
     "E = max2(E - o, Hleft - o);                 /* E(i,j) */"),
    ("F sign error (score)", "int64_t F = max2(Frow[j] - e, Hup - o);     /* F(i,j) */",
     "int64_t F = max2(Frow[j] + e, Hup - o);     /* F(i,j) */"),
    ("transposed matrix (score)",
     "int64_t H = Hdiag + S[a[i - 1] * K + b[j - 1]];\n            H = max2(H, E);\n            H = max2(H, F);\n            H = max2(H, 0);",
     "int64_t H = Hdiag + S[b[j - 1] * K + a[i - 1]];\n            H = max2(H, E);\n            H = max2(H, F);\n            H = max2(H, 0);"),
    ("dropped zero floor (score)", "            H = max2(H, 0);\n            Frow[j] = F;",
     "            Frow[j] = F;"),
    ("column-major end tie-break", "    if (i != bi) return i < bi;\n    return j < bj;",
     "    if (j != bj) return j < bj;\n    return i < bi;"),
    ("wrong diagonal index (full)", "int64_t h = AT(H, i - 1, j - 1) + S[a[i - 1] * K + b[j - 1]];",
     "int64_t h = AT(H, i - 1, j) + S[a[i - 1] * K + b[j - 1]];"),
    ("E opens with extend (full traceback)", "if (AT(E, i, j) == AT(H, i, j - 1) - o) state = 0;",
     "if (AT(E, i, j) == AT(H, i, j - 1) - e) state = 0;"),
    ("F before E (full traceback)",
     "                } else if (h == AT(E, i, j)) {\n                    state = 1;\n"
     "                } else {\n                    state = 2;",
     "                } else if (h == AT(F, i, j)) {\n                    state = 2;\n"
     "                } else {\n                    state = 1;"),
    ("extend before open (ptr)", "if (Fcur == f_open) p |= 8;", "if (Fcur == f_ext) p |= 8;"),
    ("E source mislabelled (ptr)", "else if (h == Ecur) src = 2;", "else if (h == Fcur) src = 2;"),
    ("no stop at zero (full)", "                if (h == 0) break;\n", "                if (i == 0 || j == 0) break;\n"),
    ("leading gap priced per letter (global)", "        Hrow[0] = -(o + (i - 1) * (int64_t)e);",
     "        Hrow[0] = -(i * (int64_t)e);"),
    ("semi-global top border penalised", "    return alg == 1 ? border_gap(j, o, e) : 0;",
     "    return (alg == 1 || alg == 2) ? border_gap(j, o, e) : 0;"),
    ("semi-global left border free", "    return (alg == 1 || alg == 2) ? border_gap(i, o, e) : 0;",
     "    return alg == 1 ? border_gap(i, o, e) : 0;"),
    ("overlap ends in the last row only", "        default: return i == m || j == n;",
     "        default: return i == m;"),
    ("zero floor in the variant recurrence", "            if (alg == 0) h = max2(h, 0);\n            AT(H, i, j) = h;",
     "            if (alg <= 1) h = max2(h, 0);\n            AT(H, i, j) = h;"),
    ("variant end cell: last maximum", "            if (!found || h > best) { best = h; bi = i; bj = j; found = 1; }",
     "            if (!found || h >= best) { best = h; bi = i; bj = j; found = 1; }"),
    ("global border run not forced", "                    while (i > 0) { rev[k++] = 'D'; i--; }",
     "                    i = 0;"),
    ("zero floor in the global score", "            H = max2(H, F);\n            Frow[j] = F;\n            Hdiag = Hup;\n            Hrow[j] = H;\n            Hleft = H;\n        }\n        Hrow[0]",
     "            H = max2(H, F);\n            H = max2(H, 0);\n            Frow[j] = F;\n            Hdiag = Hup;\n            Hrow[j] = H;\n            Hleft = H;\n        }\n        Hrow[0]"),
]


def _battery(lib):
    """Run the quick pins against one compiled copy; return the names that failed."""
    failed = []
    checks = [
        ("bruteforce", lambda: pins.test_bruteforce_random_small(lib, 4)),
        ("bruteforce-gappy", lambda: pins.test_bruteforce_gappy_scoring(lib)),
        ("exhaustive", lambda: pins.test_bruteforce_exhaustive_binary(lib)),
        ("symmetry", lambda: pins.test_symmetry(lib)),
        ("linear", lambda: pins.test_open_equals_extend_is_linear_gap(lib)),
        ("kadane", lambda: pins.test_huge_gaps_is_kadane(lib)),
        ("self-dna", lambda: pins.test_self_alignment_dna_closed_form(lib)),
        ("rescoring", lambda: pins.test_rescoring_medium_cases(lib)),
        ("global-bruteforce", lambda: pins.test_global_score_bruteforce(lib)),
        ("global-closed", lambda: pins.test_global_score_closed_forms(lib)),
        ("variants-bruteforce", lambda: pins.check_variants_bruteforce(lib, cases=60)),
        ("variants-closed", lambda: pins.check_variants_closed_forms(lib)),
        ("variants-rescoring", lambda: pins.check_variants_symmetry_and_rescoring(lib)),
    ]
    for name, fn in checks:
        try:
            fn()
        except Exception:  # noqa: BLE001 - any failure counts as caught
            failed.append(name)
    return failed


def test_unmutated_copy_passes_battery():
    with tempfile.TemporaryDirectory() as d:
        so = O.compile_source(O.SOURCE, os.path.join(d, "copy.so"))
        assert _battery(O.OracleLib(so)) == []


def _battery_in_child(so_path):
    """Run the battery in a fresh interpreter: a planted mistake may crash it,
    which counts as caught."""
    code = ("import json, sys; sys.path[:0] = %r; import test_oracle_mutants as T; "
            "from oracle import oracle as O; print(json.dumps(T._battery(O.OracleLib(%r))))"
            % ([os.path.dirname(os.path.abspath(__file__)),
                os.path.dirname(os.path.dirname(os.path.abspath(__file__)))], so_path))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        return ["crashed (%d)" % r.returncode]
    return json.loads(r.stdout.strip().splitlines()[-1])


# Mutants whose text also occurs in another function name that function:
# the mistake is planted in its body only.
SCOPED = {
    "wrong diagonal index (full)": "int oracle_sw_align_full(",
    "E opens with extend (full traceback)": "int oracle_sw_align_full(",
    "F before E (full traceback)": "int oracle_sw_align_full(",
    "wrong diagonal index (variants)": "int oracle_align_alg(",
    "E opens with extend (variants)": "int oracle_align_alg(",
    "F before E (variants)": "int oracle_align_alg(",
}
MUTANTS += [
    ("wrong diagonal index (variants)", "int64_t h = AT(H, i - 1, j - 1) + S[a[i - 1] * K + b[j - 1]];",
     "int64_t h = AT(H, i - 1, j) + S[a[i - 1] * K + b[j - 1]];"),
    ("E opens with extend (variants)", "if (AT(E, i, j) == AT(H, i, j - 1) - o) state = 0;",
     "if (AT(E, i, j) == AT(H, i, j - 1) - e) state = 0;"),
    ("F before E (variants)",
     "                } else if (h == AT(E, i, j)) {\n                    state = 1;\n"
     "                } else {\n                    state = 2;",
     "                } else if (h == AT(F, i, j)) {\n                    state = 2;\n"
     "                } else {\n                    state = 1;"),
]


def _plant(src, name, orig, bad):
    """The source with the mistake planted: orig must occur exactly once in
    the whole file, or, for a scoped mutant, exactly once in its function."""
    if name not in SCOPED:
        assert src.count(orig) == 1, name
        return src.replace(orig, bad)
    start = src.index(SCOPED[name])
    end = src.index("\n}\n", start)
    body = src[start:end]
    assert body.count(orig) == 1, name
    return src[:start] + body.replace(orig, bad) + src[end:]


@pytest.mark.parametrize("name,orig,bad", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(name, orig, bad):
    src = open(O.SOURCE).read()
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "mutant.c")
        with open(c, "w") as f:
            f.write(_plant(src, name, orig, bad))
        so = O.compile_source(c, os.path.join(d, "mutant.so"))
        failed = _battery_in_child(so)
    assert failed, "planted mistake %r was not caught by any pin" % name


# Planted mistakes in the Python top-k of the oracle (oracle.py), each run
# against the hand-written rankings in a module built from the mutated source.
PY_MUTANTS = [
    ("top-k ties by descending subject", "key=lambda s: (-int(scores[s]), s)",
     "key=lambda s: (-int(scores[s]), -s)"),
    ("top-k ascending score", "key=lambda s: (-int(scores[s]), s)", "key=lambda s: (int(scores[s]), s)"),
    ("top-k drops zero scores", "return [(s, int(scores[s])) for s in order[:k]]",
     "return [(s, int(scores[s])) for s in order[:k] if scores[s] > 0]"),
    ("top-k off by one", "for s in order[:k]]", "for s in order[:k + 1]]"),
]


@pytest.mark.parametrize("name,orig,bad", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_python_mutant_is_caught(name, orig, bad):
    import types
    path = os.path.join(os.path.dirname(O.SOURCE), "oracle.py")
    src = open(path).read()
    assert src.count(orig) == 1, name
    mod = types.ModuleType("oracle_mutant")
    mod.__file__ = path
    sys.modules["oracle_mutant"] = mod          # dataclasses look their module up
    try:
        exec(compile(src.replace(orig, bad), path, "exec"), mod.__dict__)
    finally:
        del sys.modules["oracle_mutant"]
    with pytest.raises(AssertionError):
        pins.check_top_k(mod.top_k)
    pins.check_top_k(O.top_k)            # the real one passes
