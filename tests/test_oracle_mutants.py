"""Mutation check of the oracle's pins.

Each case plants one plausible mistake in a COPY of the oracle's C source
(on the CPU), builds it, and runs the sampler/table pins against the
mutant in a child pytest process: every mutant must make at least one pin
fail.  The committed oracle is untouched.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "zig_oracle.c")

# (name, original text, mutated text, pins to run)
MUTANTS = [
    ("reflect_literal_appendix",  # x <- 1 - U_y, y <- U_x (not a bijection)
     "double nx = 1.0 - uy, ny = 1.0 - ux;", "double nx = 1.0 - uy, ny = ux;",
     "enumeration"),
    ("cap_dropped", "build_alias(t, A, L + 1);", "build_alias(t, A, L);",
     "enumeration or alias"),
    ("band_offset_wrong_height",  # y measured from f_j instead of f_{j-1}
     "double y = fma(uy, t->df[j], t->f[j - 1]);\n    double bound = exp(-xx);",
     "double y = fma(uy, t->df[j], t->f[j]);\n    double bound = exp(-xx);",
     "enumeration or keeps_j"),
    ("x_from_wrong_edge",
     "double xx = fma(ux, t->dX[j], t->X[j]);\n    /* Below",
     "double xx = fma(ux, t->dX[j], t->X[j - 1]);\n    /* Below",
     "enumeration or reflection"),
    ("redraw_j_on_reject",  # "go to 3" instead of keeping j
     "    ux = u64_of(t, orc_next(w));\n  }\n}",
     "    j = orc_alias_pick(t, orc_next(w)); if (j == 0) j = 1;\n    ux = u64_of(t, orc_next(w));\n  }\n}",
     "keeps_j"),
    ("tail_without_X0", "return t->X[0] + inner;", "return inner;",
     "enumeration or tail"),
    ("mt_tail_wrong_test", "if (b + b > a * a) break;", "if (b > a * a) break;",
     "marsaglia or normal_tail_law"),
    ("philox_key_bump_missing", "    k0 += PHILOX_W0;\n    k1 += PHILOX_W1;\n", "",
     "aten"),
    ("sign_bit_wrong", "int neg = (int)((w0 >> tn->ibits) & 1u);\n  double U1",
     "int neg = (int)((w0 >> 63) & 1u);\n  double U1", "fast_path"),
]


@pytest.mark.parametrize("name,orig,mut,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, orig, mut, pins):
    src = open(SRC).read()
    assert src.count(orig) == 1, f"mutation anchor for {name} not unique"
    d = tmp_path / "orc"
    d.mkdir()
    shutil.copy(os.path.join(ROOT, "oracle", "zig_oracle.h"), d / "zig_oracle.h")
    (d / "zig_oracle.c").write_text(src.replace(orig, mut))
    lib = str(d / "liborc_mutant.so")
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=gnu11",
                    str(d / "zig_oracle.c"), "-o", lib, "-lm", "-lpthread"], check=True)
    env = dict(os.environ, ZIG_ORACLE_LIB=lib)
    files = [os.path.join(ROOT, "tests", f) for f in
             ("test_oracle_sampler.py", "test_oracle_tables.py", "test_oracle_philox.py")]
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "-k", pins, *files], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert "passed" in r.stdout or "failed" in r.stdout, r.stdout[-2000:] + r.stderr[-2000:]
    assert r.returncode == 1, f"mutant {name} survived:\n" + r.stdout[-1500:]
