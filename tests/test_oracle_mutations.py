"""The oracle's pins catch the plausible mistakes: each case below plants one
mistake in a copy of the oracle (on the CPU, in a scratch folder of the
repository), rebuilds it and runs the pins in a fresh process; the run must
fail.  A pin set that let one of them through would not pin the oracle."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SCRATCH = os.path.join(ROOT, "_mutants")

MUTATIONS = [
    ("skip test flipped (Section 4.5)", "(rb[bi].r < c->hf * theta)", "(rb[bi].r > c->hf * theta)"),
    ("min for max in the block summary (Eq. summary)", "else if (v > mx[tt]) mx[tt] = v;",
     "else if (v < mx[tt]) mx[tt] = v;"),
    ("argmin clustering (Section 4.1.2)", "if (ci == 0 || s > best[i])", "if (ci == 0 || s < best[i])"),
    ("q dropped from the summary score", "r += qd[o->sterm[e]] * sv;", "r += sv;"),
    ("offset m dropped from dequantisation", "(double)o->qm[b] + (double)o->scode[e] * (double)o->qsz[b]",
     "(double)o->scode[e] * (double)o->qsz[b]"),
    ("documents scored once per list, not once per query", "if (seen[dd] == mark) continue;",
     "if (0) continue;"),
    ("alpha-MSS in ascending order", "  if (p->a > q->a) return -1;\n  if (p->a < q->a) return 1;",
     "  if (p->a < q->a) return -1;\n  if (p->a > q->a) return 1;"),
    ("alpha-MSS keeps one coordinate too many", "    if (c >= target) return i + 1;",
     "    if (c >= target) return i + 2 <= n ? i + 2 : n;"),
    ("lists keep the smallest values",
     "  if (a->v > b->v) return -1;\n  if (a->v < b->v) return 1;\n  return (a->doc > b->doc) - (a->doc < b->doc);",
     "  if (a->v < b->v) return -1;\n  if (a->v > b->v) return 1;\n  return (a->doc > b->doc) - (a->doc < b->doc);"),
    ("blocks visited in ascending score", "  if (a->r > b->r) return -1;\n  if (a->r < b->r) return 1;",
     "  if (a->r < b->r) return -1;\n  if (a->r > b->r) return 1;"),
    ("exact top-k without the query weight", "acc[dd] += qv * (double)c->L->val[e];",
     "acc[dd] += (double)c->L->val[e];"),
    ("quantisation rounds up", "floor(((double)o->sval[used + i] - (double)lo) / (double)size)",
     "ceil(((double)o->sval[used + i] - (double)lo) / (double)size)"),
    ("kappa-NN expansion reads the wrong graph row", "c->knn[(uint64_t)S[i] * c->kappa + e]",
     "c->knn[(uint64_t)(S[i] + 1) * c->kappa + e]"),
]


def run_pins(tag, old=None, new=None):
    """Copies the oracle, generator and tests, plants old -> new in the
    oracle's C source (if given), runs the pins; returns the pytest run."""
    work = os.path.join(SCRATCH, tag)
    shutil.rmtree(work, ignore_errors=True)
    os.makedirs(work)
    try:
        for d in ("oracle", "synth", "tests"):
            shutil.copytree(os.path.join(ROOT, d), os.path.join(work, d),
                            ignore=shutil.ignore_patterns("*.so", "__pycache__", "*.tmp*"))
        shutil.copy(os.path.join(ROOT, "pytest.ini"), work)
        if old is not None:
            src = os.path.join(work, "oracle", "oracle.c")
            text = open(src).read()
            assert text.count(old) == 1, "the mutation site moved"
            with open(src, "w") as f:
                f.write(text.replace(old, new))
        return subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-q", "-x",
                               "-p", "no:cacheprovider"], cwd=work, capture_output=True, text=True, timeout=900)
    finally:
        shutil.rmtree(work, ignore_errors=True)


def test_unchanged_copy_passes():
    """The harness itself: an unchanged copy passes every pin."""
    r = run_pins("control")
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_the_mistake(name, old, new):
    r = run_pins(str(MUTATIONS.index((name, old, new))), old, new)
    assert r.returncode != 0, f"{name}: every pin passed\n{r.stdout[-2000:]}"
    assert "failed" in r.stdout, r.stdout[-2000:]
