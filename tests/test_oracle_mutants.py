"""Planted mistakes in the oracle, on the CPU: each plausible slip below is
made in a copy of oracle/hav_oracle.cpp, the copy is compiled on its own, and
the pins (tests/test_oracle_pins.py, test_oracle_variants.py and
test_oracle_search.py, without their two slow whole-scene checks) run
against it.  Every mutant must fail at least one pin; a mutant that
passes would mean the pins cannot tell that slip from the paper's method.
The oracle itself is untouched: the copy is loaded through HAV_ORACLE_LIB."""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "hav_oracle.cpp")

# (what the slip breaks, text of the oracle, the slip); the first occurrence
# of the text is replaced
MUTANTS = [
    ("Eq. 2: round instead of floor", "float f = std::floor(q);", "float f = std::round(q);"),
    ("Sec. 3.2: corner instead of centre (dropped + 0.5)", "float half = f[a] + 0.5f;", "float half = f[a];"),
    ("Sec. 3.2: squared distance without z", "return xy + zz;", "return xy;"),
    ("Sec. 3.2: farthest instead of closest point",
     "else if (packed < it->second) it->second = packed;", "else if (packed > it->second) it->second = packed;"),
    ("Sec. 3.3: too many voxels lowers hi",
     "            if (K > k_max) {\n                lo = s;", "            if (K > k_max) {\n                hi = s;"),
    ("Sec. 3.3: K == m_l not accepted",
     "} else if (K < m_l) {\n                hi = s;", "} else if (K <= m_l) {\n                hi = s;"),
    ("Sec. 3.3: K == (1 + sigma) m_l not accepted",
     "            if (K > k_max) {\n                lo = s;", "            if (K >= k_max) {\n                lo = s;"),
    ("Sec. 3.3: tolerance sigma dropped",
     "const int64_t k_max = m_l + (m_l * p->sigma_num) / p->sigma_den;", "const int64_t k_max = m_l;"),
    ("Sec. 3.3: midpoint misparenthesised", "else s = (lo + hi) * 0.5f;", "else s = lo + hi * 0.5f;"),
    ("Sec. 3.3: bracket from the smallest extent",
     "s_hi = std::max(s_hi, t);", "s_hi = (a == 0) ? t : std::min(s_hi, t);"),
    ("Sec. 3.3: unfinished search takes hi", "if (!accepted) s_star = (lo > 0.0f) ? lo : hi;",
     "if (!accepted) s_star = hi;"),
    ("cut-off keeps the largest priorities", "std::sort(pr.begin(), pr.end());",
     "std::sort(pr.rbegin(), pr.rend());"),
    ("cut-off priority: SplitMix64 constant", "0xBF58476D1CE4E5B9ull", "0xBF58476D1CE4E5B8ull"),
    ("shortfall filled from the highest index",
     "            for (int32_t i : active) {\n                if (need == 0) break;",
     "            for (auto it2 = active.rbegin(); it2 != active.rend(); ++it2) {\n"
     "                const int32_t i = *it2;\n                if (need == 0) break;"),
    ("Eq. 3: layer budgets in reverse order", "ml[l] = (m * w[l]) / S;", "ml[l] = (m * w[layers - 1 - l]) / S;"),
    ("Eq. 3: points taken by a coarser layer re-enter",
     "if (!taken[i]) active.push_back(static_cast<int32_t>(i));", "active.push_back(static_cast<int32_t>(i));"),
    ("Eq. 2: aspect ratio on the wrong axis", "v[a] = s * c.r[a];", "v[a] = s * c.r[(a + 1) % 3];"),
    ("level chain: indices of the level, not of the cloud",
     "out_concat[off + r] = orig[i];", "out_concat[off + r] = i;"),
    # Table 6 variants, the comparators and the guided start
    ("Table 6 mean: divided by count + 1", "/ static_cast<double>(acc.count);",
     "/ static_cast<double>(acc.count + 1);"),
    ("Table 6 centre: the voxel corner", "const float cen = acc.f[a] + 0.5f;", "const float cen = acc.f[a];"),
    ("Table 6 random: SplitMix64 draw counter off by one", "(counter + 1) * 0x9E3779B97F4A7C15ull",
     "counter * 0x9E3779B97F4A7C15ull"),
    ("Table 6 random: low word of the draw",
     "hi32 = static_cast<uint32_t>(random_draw(p->seed, uint64_t(i)) >> 32);",
     "hi32 = static_cast<uint32_t>(random_draw(p->seed, uint64_t(i)));"),
    ("Table 6 fixed voxel: the size ignored", "if (fixed) s_star = p->fixed_s;", "if (fixed) s_star = c.s_hi;"),
    ("Fig. 3 spacing: a point is its own neighbour", "            if (q == r) continue;\n", ""),
    ("grouping: radius inclusive", "if (d2 < r2) row[cnt++]", "if (d2 <= r2) row[cnt++]"),
    ("grouping: padded with the last index", "for (int32_t s = cnt; s < nsample; ++s) row[s] = row[0];",
     "for (int32_t s = cnt; s < nsample; ++s) row[s] = row[cnt - 1];"),
    ("Eq. 1 FPS: ties to the highest index", "if (best[i] > bestd) { bestd = best[i]; arg = i; }",
     "if (best[i] >= bestd) { bestd = best[i]; arg = i; }"),
    ("Eq. 1 FPS: distance to the last pick only", "if (d2 < best[i]) best[i] = d2;", "best[i] = d2;"),
    ("guided start: budget ratio without the square root", "g = guide->s * std::sqrt(ratio);",
     "g = guide->s * ratio;"),
    ("guided start: first guess without the square root", "g = c.s_hi / std::sqrt(static_cast<float>(m_l));",
     "g = c.s_hi / static_cast<float>(m_l);"),
    ("guided start: doubling up to the top itself", "else if (up && lo * 2.0f < hi) s = lo * 2.0f;",
     "else if (up && lo * 2.0f <= hi) s = lo * 2.0f;"),
    ("guided start: doubling again after a low count", "                hi = s;\n                up = false;",
     "                hi = s;"),
]


def _run_mutant(tmp, k, old, new, src):
    d = os.path.join(tmp, f"m{k}")
    os.makedirs(d)
    with open(os.path.join(d, "o.cpp"), "w") as f:
        f.write(src.replace(old, new, 1))
    lib = os.path.join(d, "libo.so")
    subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                    "-o", lib, os.path.join(d, "o.cpp")], check=True, capture_output=True)
    env = dict(os.environ, HAV_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "tests/test_oracle_variants.py",
                        "tests/test_oracle_search.py", "-x", "-q", "-p", "no:cacheprovider",
                        "-k", "not output_invariants and not exact_at_scale"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode


def test_every_planted_mistake_fails_a_pin(tmp_path):
    with open(SRC) as f:
        src = f.read()
    for what, old, new in MUTANTS:
        assert old in src, f"the oracle no longer contains the text of {what!r}"
    workers = max(1, min(8, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(workers) as ex:
        rcs = list(ex.map(lambda a: _run_mutant(str(tmp_path), a[0], a[1][1], a[1][2], src),
                          enumerate(MUTANTS)))
    # exit code 1: some pin failed; 0 would mean the pins passed the mistake
    survivors = [what for (what, _, _), rc in zip(MUTANTS, rcs) if rc != 1]
    assert not survivors, f"mistakes no pin catches (or that did not run): {survivors}"


@pytest.mark.parametrize("what,old,new", MUTANTS[:1])
def test_the_clean_copy_passes(tmp_path, what, old, new):
    # the same machinery with no slip planted passes every pin
    with open(SRC) as f:
        src = f.read()
    assert _run_mutant(str(tmp_path), 0, old, old, src) == 0
