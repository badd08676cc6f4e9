"""The oracle's pins catch the plausible mistakes: each case below plants one
mistake in a copy of the oracle (on the CPU, in pytest's temporary folder),
rebuilds it and runs the pins in a fresh process; the run must fail.  A pin
set that let one of them through would not pin the oracle."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PIN_FILES = ("tests/test_oracle_pins.py", "tests/test_oracle_mlp.py")

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
    ("list ties at the cut go to the higher document id (reading R2)",
     "  if (a->v < b->v) return 1;\n  return (a->doc > b->doc) - (a->doc < b->doc);",
     "  if (a->v < b->v) return 1;\n  return (a->doc < b->doc) - (a->doc > b->doc);"),
    ("blocks visited in ascending score", "  if (a->r > b->r) return -1;\n  if (a->r < b->r) return 1;",
     "  if (a->r < b->r) return -1;\n  if (a->r > b->r) return 1;"),
    ("exact top-k without the query weight", "acc[dd] += qv * (double)c->L->val[e];",
     "acc[dd] += (double)c->L->val[e];"),
    ("quantisation rounds up", "floor(((double)o->sval[used + i] - (double)lo) / (double)size)",
     "ceil(((double)o->sval[used + i] - (double)lo) / (double)size)"),
    ("kappa-NN expansion reads the wrong graph row", "c->knn[(uint64_t)S[i] * c->kappa + e]",
     "c->knn[(uint64_t)(S[i] + 1) * c->kappa + e]"),
    ("graph refinement skips u's own list", "for (uint32_t i = 0; i <= K; i++) {",
     "for (uint32_t i = 1; i <= K; i++) {"),
    ("graph refinement keeps u among its own candidates", "st[ui] = mark; /* u itself is never a candidate */",
     "st[ui] = 0; /* u itself is never a candidate */"),
    ("pair scoring keeps the previous query's terms",
     "for (uint64_t p = qip[cur]; p < qip[cur + 1]; p++) qd[qt[p]] = 0.0;",
     "for (uint64_t p = qip[cur]; p < qip[cur]; p++) qd[qt[p]] = 0.0;"),
]

# mistakes in the oracle MLP (oracle/mlp.py); each is a list of (old, new)
# sites.  The first is shared by the forward pass and the gradient, so the
# finite-difference pin alone would not see it.
MLP_MUTATIONS = [
    ("absolute value for ReLU in forward and gradient",
     [("a1 = np.maximum(z1, 0.0)", "a1 = np.abs(z1)"), ("* (z1 > 0)", "* np.sign(z1)")]),
    ("hidden layers without biases", [("z1 = x @ p[\"W1\"].T + p[\"b1\"]", "z1 = x @ p[\"W1\"].T")]),
]


def run_pins(work, fname=None, sites=()):
    """Copies the oracle, generator and tests into `work`, plants each
    (old, new) site in oracle/<fname>, runs the pins; returns the pytest run."""
    for d in ("oracle", "synth", "tests"):
        shutil.copytree(os.path.join(ROOT, d), os.path.join(work, d),
                        ignore=shutil.ignore_patterns("*.so", "__pycache__", "*.tmp*"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), work)
    if sites:
        src = os.path.join(work, "oracle", fname)
        text = open(src).read()
        for old, new in sites:
            assert text.count(old) >= 1, "the mutation site moved"
            text = text.replace(old, new)
        with open(src, "w") as f:
            f.write(text)
    return subprocess.run([sys.executable, "-m", "pytest", *PIN_FILES, "-q", "-x", "-p", "no:cacheprovider"],
                          cwd=work, capture_output=True, text=True, timeout=900)


def test_unchanged_copy_passes(tmp_path):
    """The harness itself: an unchanged copy passes every pin."""
    r = run_pins(str(tmp_path))
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_the_mistake(tmp_path, name, old, new):
    r = run_pins(str(tmp_path), "oracle.c", [(old, new)])
    assert r.returncode != 0, f"{name}: every pin passed\n{r.stdout[-2000:]}"
    assert "failed" in r.stdout, r.stdout[-2000:]


@pytest.mark.parametrize("name,sites", MLP_MUTATIONS, ids=[m[0] for m in MLP_MUTATIONS])
def test_pins_catch_the_mlp_mistake(tmp_path, name, sites):
    r = run_pins(str(tmp_path), "mlp.py", sites)
    assert r.returncode != 0, f"{name}: every pin passed\n{r.stdout[-2000:]}"
    assert "failed" in r.stdout, r.stdout[-2000:]
