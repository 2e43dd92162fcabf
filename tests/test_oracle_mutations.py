"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (a flipped
sign, a wrong index, a dropped term, a changed tie rule), builds it with gcc
on the CPU, and runs the oracle pin tests against that copy: at least one pin
must fail.  Nothing here touches the CUDA path.
"""
import glob
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "askit_oracle.c")

MUTATIONS = [
    ("householder sign", "double beta = (alpha >= 0.0) ? -nrm : nrm;", "double beta = (alpha >= 0.0) ? nrm : -nrm;"),
    ("pivot tie rule", "if (acc > best) { best = acc; p = j; }", "if (acc >= best) { best = acc; p = j; }"),
    ("skeleton weights drop P term", "t->wsk[a][q * r + z] = v[(size_t)t->piv[a][q] * r + z] + acc;",
     "t->wsk[a][q * r + z] = v[(size_t)t->piv[a][q] * r + z];"),
    ("evaluate skips right child",
     "evaluate_rec(t, x, pset, np, 2 * a + 1, depth + 1, u, near, far, part, far_height);", ""),
    ("far height off by one", "if (far_height >= 0 && t->L - depth > far_height) pruned = 0;",
     "if (far_height >= 0 && t->L - depth >= far_height) pruned = 0;"),
    ("adaptive kappa keeps the first failing neighbor", "if (arg < cut) ki = z + 1;", "if (arg <= cut) ki = z + 2;"),
    ("distance pruning ignores the radius scale", "> rs2 * r2[a]) return v;", "> r2[a]) return v;"),
    ("neighbor pruning visits one child", "return v + visit_knn(L, 2 * a, depth + 1, pset, np) + visit_knn(L, 2 * a + 1, depth + 1, pset, np);",
     "return v + visit_knn(L, 2 * a, depth + 1, pset, np);"),
    ("centroid over half the node", "for (int64_t q = 0; q < size[a]; ++q) {\n            const float *x",
     "for (int64_t q = 0; q < size[a] / 2; ++q) {\n            const float *x"),
    ("prune test off by a level", "if ((pset[q] >> (t->L - depth)) == a) pruned = 0;",
     "if ((pset[q] >> (t->L - depth + 1)) == a) pruned = 0;"),
    ("median side", "int64_t nl = (n + 1) / 2;", "int64_t nl = n / 2;"),
    ("center", "xc[k] = acc / (double)n;", "xc[k] = acc / (double)(n + 1);"),
    ("back substitution transposed", "acc = acc - A[(size_t)i * cols + t] * P[(size_t)t * nr + j];",
     "acc = acc - A[(size_t)t * cols + i] * P[(size_t)t * nr + j];"),
    ("sampler forgets N_a", "for (int64_t q = 0; q < nr && !seen; ++q) seen = (t->trows[a][q] == j);",
     "for (int64_t q = t->nl_cnt[a]; q < nr && !seen; ++q) seen = (t->trows[a][q] == j);"),
    ("node list key sign", "cand[n].j = j; cand[n].key = t->nl_key[ch[c]][q]; ++n;",
     "cand[n].j = j; cand[n].key = -t->nl_key[ch[c]][q]; ++n;"),
    ("rp direction bits", "v[k] = ((w >> (k & 63)) & 1) ? -1.0 : 1.0;", "v[k] = ((w >> (k & 31)) & 1) ? -1.0 : 1.0;"),
    ("ID bandwidth squared", "double arg = (t->prm.kscale * D) / (h * h);", "double arg = (t->prm.kscale * D) / (h);"),
    ("direct sum drops self", "U[(size_t)t * r + q] = U[(size_t)t * r + q] + k * W[(size_t)j * r + q];",
     "if (Y || j != tgt[t]) U[(size_t)t * r + q] = U[(size_t)t * r + q] + k * W[(size_t)j * r + q];"),
    ("exp reduction tail sign", "double r = (a - n * LN2_HEAD) - n * LN2_TAIL;", "double r = (a - n * LN2_HEAD) + n * LN2_TAIL;"),
    ("exp polynomial term", "0x1.5555555555555p-3,", "0x1.5555555555555p-2,"),
    ("leaf-grouped set takes the target's neighbors",
     "for (int z = 0; z < kp; ++z) pset[np++] = t->leafof[t->knn[(size_t)p * kappa + z]];",
     "for (int z = 0; z < kp; ++z) pset[np++] = t->leafof[t->knn[(size_t)i * kappa + z]];"),
]


@pytest.mark.parametrize("name,before,after", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(name, before, after, tmp_path):
    src = open(SRC).read()
    assert before in src, name
    c = tmp_path / "mut.c"
    so = tmp_path / "mut.so"
    c.write_text(src.replace(before, after, 1))
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                           "-o", str(so), str(c), "-lm"])
    pins = sorted(p for p in glob.glob(os.path.join(HERE, "test_oracle_*.py"))
                  if not p.endswith("test_oracle_mutations.py"))
    res = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", *pins],
                         env=dict(os.environ, ASKIT_ORACLE_LIB=str(so)), capture_output=True, text=True,
                         cwd=os.path.dirname(HERE), timeout=600)
    assert res.returncode != 0, f"mistake '{name}' not caught:\n{res.stdout[-500:]}"
