"""The oracle's pins catch plausible mistakes planted in the oracle.

Each case copies the oracle's source, changes one spot into a mistake of
the kind that slips into such code (a flipped comparison, an off-by-one
bound, a dropped term, a confused index, a transposed layout), builds the
copy on its own and runs the pin tests against it in a child process: at
least one pin must fail (or the copy must crash or hang there).  A mistake
that every pin lets through marks a hole in the pins.  The oracle itself is
never modified; the copies live in a temporary folder.
"""
import os
import subprocess
import sys
import textwrap
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_C = os.path.join(ROOT, "oracle", "oracle.c")
LEARNED_PY = os.path.join(ROOT, "oracle", "learned.py")
ORDERING_PY = os.path.join(ROOT, "oracle", "ordering.py")

# (name, text in the oracle, replacement, replace every occurrence)
C_MUTANTS = [
    # core numbers (Batagelj-Zaversnik)
    ("cores-lower-equal-degree", "if (deg[u] > deg[v]) {", "if (deg[u] >= deg[v]) {", False),
    ("cores-degree-never-lowered", "        bin[du]++;\n        deg[u]--;", "        bin[du]++;", False),
    # greedy colouring
    ("colours-start-at-two", "    int32_t c = 1;\n    while (mark[c] == i) c++;",
     "    int32_t c = 2;\n    while (mark[c] == i) c++;", False),
    ("colours-ignore-neighbours", "if (c > 0 && c <= n + 1) mark[c] = i;", "if (c > 0 && c <= n + 1) mark[c] = i - 1;", False),
    # Algorithm 1
    ("heuristic-C-starts-empty",
     "    C[c++] = v;\n    for (int64_t j = 0; j < ns; j++) {\n      int32_t u = S[j].v, ok = 1;\n"
     "      for (int32_t t = 0; t < c && ok; t++) ok = adjacent(rp,",
     "    for (int64_t j = 0; j < ns; j++) {\n      int32_t u = S[j].v, ok = 1;\n"
     "      for (int32_t t = 0; t < c && ok; t++) ok = adjacent(rp,", False),
    ("heuristic-increasing-core", "if (a->k != b->k) return a->k > b->k ? -1 : 1;",
     "if (a->k != b->k) return a->k < b->k ? -1 : 1;", False),
    ("heuristic-smaller-degree-first", "if (a->d != b->d) return a->d > b->d ? -1 : 1;",
     "if (a->d != b->d) return a->d < b->d ? -1 : 1;", False),
    ("heuristic-larger-id-first", "return (a->v > b->v) - (a->v < b->v);", "return (a->v < b->v) - (a->v > b->v);", False),
    ("heuristic-skip-at-equal-core", "if (mode == 0 && core[v] < max) continue;", "if (mode == 0 && core[v] <= max) continue;", False),
    ("heuristic-skips-last-member", "for (int32_t t = 0; t < c && ok; t++) ok = adjacent(rp,",
     "for (int32_t t = 0; t + 1 < c && ok; t++) ok = adjacent(rp,", False),
    ("heuristic-strict-candidate-filter", "if (core[u] >= T) {", "if (core[u] > T) {", False),
    ("heuristic-mode1-ties-to-largest", "(mode == 1 && c == max && v < best_v)", "(mode == 1 && c == max && v > best_v)", False),
    # Algorithm 2
    ("prune-strict", "newid[v] = (K0[v] >= hs)", "newid[v] = (K0[v] > hs)", False),
    ("initialbranch-core-test-off-by-one", "if (KP + 1 <= s->hsize) goto done;", "if (KP + 1 <= s->hsize + 1) goto done;", False),
    ("initialbranch-neighbourhood-core-strict", "if (kn[a] >= s->hsize)", "if (kn[a] > s->hsize)", True),
    ("initialbranch-colour-bound-off-by-one", "if (L <= s->hsize) goto done;", "if (L <= s->hsize + 1) goto done;", False),
    ("initialbranch-u-left-out", "    if (!inserted && w > u) { s->P[np++] = u; inserted = 1; }\n",
     "    if (!inserted && w > u) { inserted = 1; }\n", False),
    ("branch-colour-bound-off-by-one", "if (csize + cu <= s->hsize) break;", "if (csize + cu <= s->hsize + 1) break;", False),
    ("branch-picks-smallest-colour",
     "if (colors[i] >= colors[at]) at = i;\n    int32_t u = idx[at], cu = colors[at];\n"
     "    for (int32_t i = at; i + 1 < cnt; i++) { idx[i] = idx[i + 1]; colors[i] = colors[i + 1]; }\n"
     "    cnt--;\n    if (csize + cu <= s->hsize)",
     "if (colors[i] <= colors[at]) at = i;\n    int32_t u = idx[at], cu = colors[at];\n"
     "    for (int32_t i = at; i + 1 < cnt; i++) { idx[i] = idx[i + 1]; colors[i] = colors[i + 1]; }\n"
     "    cnt--;\n    if (csize + cu <= s->hsize)", False),
    ("branch-P-index-as-vertex", "&& alive(s, s->P[w])) pidx[np2++] = w;", "&& alive(s, w)) pidx[np2++] = w;", False),
    ("branch-no-adjacency-filter", "if (s->adj[(int64_t)u * s->np + w] && alive(s, s->P[w]))", "if (alive(s, s->P[w]))", False),
    ("branch-witness-from-P-index", "s->H[i] = s->orig[s->P[s->C[i]]];", "s->H[i] = s->orig[s->C[i]];", False),
    ("branch-incumbent-not-raised", "      s->hsize = c2;\n", "", False),
    ("search-implicit-removal-off-by-one", "K2[byk[kptr]] < s.hsize", "K2[byk[kptr]] <= s.hsize", False),
    ("small-cores-no-running-max", "if (deg[at] > k) k = deg[at];", "k = deg[at];", False),
    # shared helpers
    ("adjacency-search-overshoots", "if (ci[mid] < b) lo = mid + 1; else hi = mid;",
     "if (ci[mid] <= b) lo = mid + 1; else hi = mid;", False),
    ("is-clique-skips-a-pair", "for (int32_t j = i + 1; j < k; j++) {", "for (int32_t j = i + 2; j < k; j++) {", False),
    # the threaded search (Section 4.5)
    ("threads-heuristic-C-starts-empty", "    C[c++] = v;\n    for (int64_t j = 0; j < ns; j++) {\n      int32_t u = S[j].v, ok = 1;\n"
     "      for (int32_t t = 0; t < c && ok; t++) ok = adjacent(h->rp,",
     "    for (int64_t j = 0; j < ns; j++) {\n      int32_t u = S[j].v, ok = 1;\n"
     "      for (int32_t t = 0; t < c && ok; t++) ok = adjacent(h->rp,", False),
    ("threads-heuristic-skips-last-member", "for (int32_t t = 0; t < c && ok; t++) ok = adjacent(h->rp,",
     "for (int32_t t = 0; t + 1 < c && ok; t++) ok = adjacent(h->rp,", False),
    ("threads-heuristic-stops-at-equal-core", "if (h->core[v] < T) break;", "if (h->core[v] <= T) break;", False),
    ("threads-prune-strict", "if (K0[order[i]] >= hs) newid", "if (K0[order[i]] > hs) newid", False),
    ("threads-root-filter-strict", "if (sh->K[sh->oci[e]] >= h) w->P[np++]", "if (sh->K[sh->oci[e]] > h) w->P[np++]", False),
    ("threads-root-size-test-off-by-one", "if (np + 1 <= h) return;", "if (np + 1 <= h + 1) return;", False),
    ("threads-adjacency-one-direction", "        w->adj[(int64_t)(b - 1) * np + a] = 1;\n", "", False),
    ("threads-neighbourhood-core-strict", "if (kn[a] + 1 >= h)", "if (kn[a] + 1 > h)", False),
    ("threads-kept-count-off-by-one", "if (cnt + 1 <= h) return;", "if (cnt + 1 <= h + 1) return;", False),
    ("threads-colour-test-without-u", "if (1 + L <= th_best(w)) return;", "if (L <= th_best(w)) return;", False),
    ("threads-branch-colour-bound-off-by-one", "if (csize + cu <= th_best(w)) break;",
     "if (csize + cu <= th_best(w) + 1) break;", False),
    ("threads-branch-no-adjacency-filter", "      if (w->adj[(int64_t)u * w->np + idx[i]]) pidx[np2++] = idx[i];",
     "      pidx[np2++] = idx[i];", False),
    ("threads-clique-member-as-index", "w->C[csize] = w->P[u];", "w->C[csize] = u;", False),
    ("threads-witness-in-new-ids", "sh->H[i] = sh->orig[w->C[i]];", "sh->H[i] = w->C[i];", False),
    ("threads-incumbent-not-published", "    __atomic_store_n(&sh->best, size, __ATOMIC_RELEASE);\n", "", False),
    ("threads-branch-coloured-in-rank-order",
     "static int cmp_knkey_id(const void *x, const void *y) {\n  const knkey *a = (const knkey *)x, *b = (const knkey *)y;\n"
     "  return (a->id > b->id) - (a->id < b->id);",
     "static int cmp_knkey_id(const void *x, const void *y) {\n  const knkey *a = (const knkey *)x, *b = (const knkey *)y;\n"
     "  return (a->i > b->i) - (a->i < b->i);", False),
    # the partitioned search
    ("part-searches-the-other-roots", "if (sh->opos[u] % sh->part_count != sh->part_rank) return;",
     "if (sh->opos[u] % sh->part_count == sh->part_rank) return;", False),
    ("part-order-not-checked", "if (later > K[v]) return 0;", "if (later > K[v] + 1000000) return 0;", False),
]

PY_MUTANTS = [
    ("bf16-truncates", "(a + 0x7FFF + ((a >> 16) & 1)) >> 16", "a >> 16", False),
    ("bf16-ties-away", "(a + 0x7FFF + ((a >> 16) & 1)) >> 16", "(a + 0x8000) >> 16", False),
    ("features-strict-core-filter", "qual = nb[core[nb] >= core[v]]", "qual = nb[core[nb] > core[v]]", False),
    ("features-degree-for-count", "out[v, 5] = np.log1p(c) / ldmax", "out[v, 5] = np.log1p(d) / ldmax", False),
    ("features-Q-without-core-filter", "Q = qual[:T].tolist()", "Q = nb[:T].tolist()", False),
    ("features-Q-last-neighbours", "Q = qual[:T].tolist()", "Q = qual[-T:].tolist()", False),
    ("features-triangles-counted-twice", "t = sum(1 for i in range(q) for j in range(i + 1, q) if adj[i][j])",
     "t = sum(1 for i in range(q) for j in range(q) if i != j and adj[i][j])", False),
    ("features-colouring-ignores-edges", "used = {col[j] for j in range(i) if adj[i][j]}",
     "used = {col[j] for j in range(i) if not adj[i][j]}", False),
    ("features-bound-without-v", "out[v, 3] = (chi + 1) / (T + 1)", "out[v, 3] = chi / (T + 1)", False),
    ("features-density-not-count", "out[v, 2] = t / (T * (T - 1) / 2)",
     "out[v, 2] = t / max(q * (q - 1) / 2, 1)", False),
    ("w1-transposed", "W1 = w[OFF_W1:OFF_B1].reshape(H, F)", "W1 = w[OFF_W1:OFF_B1].reshape(F, H).T", False),
    ("w2-transposed", "W2 = w[OFF_W2:OFF_B2].reshape(H, H)", "W2 = w[OFF_W2:OFF_B2].reshape(H, H).T", False),
    ("biases-rounded-to-bf16", "    b1 = p[OFF_B1:OFF_W2]\n", "    b1 = w[OFF_B1:OFF_W2]\n", False),
    ("no-relu-layer-2", "    h2 = np.maximum(h1 @ W2.T + b2, 0.0)\n    return", "    h2 = h1 @ W2.T + b2\n    return", False),
    ("no-output-bias", "    return h2 @ w3 + b3\n", "    return h2 @ w3\n", False),
    ("loss-sign", "np.logaddexp(0.0, s) - y * s", "np.logaddexp(0.0, s) + y * s", False),
    ("loss-weights-swapped", "    w = np.where(y > 0.5, pos_weight, 1.0)\n    return",
     "    w = np.where(y > 0.5, 1.0, pos_weight)\n    return", False),
    ("loss-sum-not-mean", "return float(np.mean(w * (np.logaddexp(0.0, s) - y * s)))",
     "return float(np.sum(w * (np.logaddexp(0.0, s) - y * s)))", False),
    ("grad-relu-mask-layer-1", "d1 = (d2 @ W2) * (z1 > 0)", "d1 = (d2 @ W2) * (z1 >= -1e30)", False),
    ("grad-w2-transposed", "g[OFF_W2:OFF_B2] = (d2.T @ h1).ravel()", "g[OFF_W2:OFF_B2] = (h1.T @ d2).ravel()", False),
    ("grad-backprop-through-W2-transposed", "d1 = (d2 @ W2) * (z1 > 0)", "d1 = (d2 @ W2.T) * (z1 > 0)", False),
    ("grad-missing-mean", "gs = w * (1.0 / (1.0 + np.exp(-s)) - y) / n", "gs = w * (1.0 / (1.0 + np.exp(-s)) - y)", False),
    ("grad-b1-dropped", "    g[OFF_B1:OFF_W2] = d1.sum(axis=0)\n", "", False),
    ("adam-no-bias-correction", "    mhat = m / (1.0 - beta1 ** t)\n", "    mhat = m\n", False),
    ("adam-second-moment-uncorrected", "    vhat = v / (1.0 - beta2 ** t)\n", "    vhat = v\n", False),
    ("adam-betas-swapped", "    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g\n",
     "    m = beta2 * np.asarray(m, dtype=np.float64) + (1.0 - beta2) * g\n", False),
    ("adam-eps-inside-root", "(np.sqrt(vhat) + eps)", "np.sqrt(vhat + eps)", False),
]


ORDERING_MUTANTS = [
    ("order-ties-by-id-not-rank", "k = (len(c), -int(rank[v]))\n            for u in c:",
     "k = (len(c), -v)\n            for u in c:", False),
    ("order-candidates-by-id", "cand.sort(key=lambda u: (-int(core[u]), -int(deg[u]), u))", "cand.sort()", False),
    ("order-candidates-by-degree-first", "cand.sort(key=lambda u: (-int(core[u]), -int(deg[u]), u))",
     "cand.sort(key=lambda u: (-int(deg[u]), -int(core[u]), u))", False),
    ("order-accept-checks-start-only", "if all(best[u] == k for u in c):", "if best[v] == k:", False),
    ("order-members-ascending-degree", "order.extend(sorted(c, key=lambda u: (-int(deg[u]), u)))",
     "order.extend(sorted(c, key=lambda u: (int(deg[u]), u)))", False),
    ("order-members-by-id", "order.extend(sorted(c, key=lambda u: (-int(deg[u]), u)))", "order.extend(sorted(c))", False),
    ("order-dead-candidates-kept", "cand = [u for u in rows[v].tolist() if alive[u]]",
     "cand = [u for u in rows[v].tolist()]", False),
    ("order-cliques-by-size", "        for v in sorted(cl):", "        for v in sorted(cl, key=lambda v: -len(cl[v])):", False),
    ("gap-from-zero", "gaps[0] = abs(r[0] - pos[v])", "gaps[0] = r[0]", False),
    ("gap-bits-log-gap", "np.log2(1.0 + gaps)", "np.log2(np.maximum(gaps, 1))", False),
    ("gap-unsorted-row", "r = np.sort(pos[g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]]])",
     "r = pos[g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]]]", False),
]


def _mutate(src, old, new, every):
    count = src.count(old)
    assert count >= 1, "mutation site not found: %r" % old
    if not every:
        assert count == 1, "mutation site not unique: %r" % old
    return src.replace(old, new)


def _run(script, timeout=180):
    """Exit status of the pin run in a child process ('hang' on timeout)."""
    try:
        r = subprocess.run([sys.executable, "-c", script], cwd=ROOT, capture_output=True, text=True,
                           timeout=timeout)
    except subprocess.TimeoutExpired:
        return "hang", ""
    return r.returncode, (r.stdout + r.stderr)[-2000:]


PYTEST_ARGS = '["-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu", %s]'


def _c_case(tmp, name, old, new, every):
    src = _mutate(open(ORACLE_C).read(), old, new, every)
    c = os.path.join(tmp, name + ".c")
    so = os.path.join(tmp, name + ".so")
    with open(c, "w") as f:
        f.write(src)
    subprocess.run(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-pthread", c, "-o", so,
                    "-lm"], check=True)
    script = textwrap.dedent("""
        import ctypes, sys
        sys.path.insert(0, %r)
        import oracle
        oracle._lib = oracle.configure(ctypes.CDLL(%r))
        import pytest
        sys.exit(pytest.main(%s))
    """) % (ROOT, so, PYTEST_ARGS % repr(os.path.join("tests", "test_oracle.py")))
    return name, _run(script)


def _py_case(tmp, name, old, new, every, module="learned", tests="test_learned_oracle.py"):
    src = _mutate(open(os.path.join(ROOT, "oracle", module + ".py")).read(), old, new, every)
    path = os.path.join(tmp, name + ".py")
    with open(path, "w") as f:
        f.write(src)
    script = textwrap.dedent("""
        import importlib.util, sys
        sys.path.insert(0, %r)
        import oracle
        spec = importlib.util.spec_from_file_location("oracle.%s", %r)
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
        sys.modules["oracle.%s"] = mod
        setattr(oracle, %r, mod)
        import pytest
        sys.exit(pytest.main(%s))
    """) % (ROOT, module, path, module, module, PYTEST_ARGS % repr(os.path.join("tests", tests)))
    return name, _run(script)


def _ord_case(tmp, name, old, new, every):
    return _py_case(tmp, name, old, new, every, "ordering", "test_ordering_oracle.py")


def test_unmutated_copies_pass(tmp_path):
    """The harness itself: an unchanged copy passes every pin."""
    rc, tail = _c_case(str(tmp_path), "identity_c", "#include <stdint.h>", "#include <stdint.h>", False)[1]
    assert rc == 0, tail
    rc, tail = _py_case(str(tmp_path), "identity_py", "import numpy as np", "import numpy as np", False)[1]
    assert rc == 0, tail
    rc, tail = _ord_case(str(tmp_path), "identity_ord", "import numpy as np", "import numpy as np", False)[1]
    assert rc == 0, tail


@pytest.mark.parametrize("kind", ["c", "py", "ord"])
def test_every_planted_mistake_is_caught(tmp_path, kind):
    cases, fn = {"c": (C_MUTANTS, _c_case), "py": (PY_MUTANTS, _py_case), "ord": (ORDERING_MUTANTS, _ord_case)}[kind]
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        results = list(ex.map(lambda m: fn(str(tmp_path), *m), cases))
    # pytest exit 1: a pin failed; a negative status: the copy crashed; 2-5
    # would be a usage or collection error of the harness, not a catch
    broken = ["%s: %s" % (name, tail) for name, (rc, tail) in results if rc in (2, 3, 4, 5)]
    assert not broken, broken
    survivors = [name for name, (rc, _) in results if rc == 0]
    assert not survivors, "mistakes no pin catches: %s" % survivors
