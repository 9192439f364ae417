"""The range-query tree's grouping rule and level capacities, on the CPU.

The run-start test of the tree build (`tg_cpl`, `tg_start` in
csrc/hac_core.cu) is compiled here as host code, straight from the kernel
source, and run on keys staged the way the build stages them (32 empty
slots on each side of a block).  Its runs must be exactly the largest cells
of the 96-bit key hierarchy (instance number, then Morton key) that hold at
most 32 elements, with more than 32 equal keys cut every 32 positions; this
is checked against a brute-force definition on random sorted keys with
clusters, duplicates and instance boundaries.  `tree_caps` (hac_internal.cuh)
is checked for the properties the build relies on: the last level holds at
most 32 nodes, a level cut into fixed runs of 32 always fits the next
capacity, and the level count stays within the per-warp stack."""
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2106_04727_gb300", "csrc")
CXX = shutil.which("g++") or shutil.which("c++")


def _between(text, start, end):
    a = text.index(start)
    return text[a:text.index(end, a)]


def _harness(tmp_path):
    core = open(os.path.join(CSRC, "hac_core.cu")).read()
    internal = open(os.path.join(CSRC, "hac_internal.cuh")).read()
    rule = _between(core, "__device__ __forceinline__ int tg_cpl(", "// elements of level L")
    rule = rule.replace("__device__ __forceinline__", "static inline").replace(
        "__device__", "static")
    caps = _between(internal, "__host__ __device__ inline int tree_caps(", "// tinfo entries")
    caps = caps.replace("__host__ __device__ inline", "static inline")
    maxlev = re.search(r"constexpr int MAXLEV = (\d+);", internal).group(1)
    tg_h = re.search(r"constexpr int TG_H = (\d+);", core).group(1)
    src = f"""#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <vector>
constexpr int FAN = 32;
constexpr int MAXLEV = {maxlev};
constexpr int TG_H = {tg_h};
constexpr int TPB = 256;
static int __clz(int x) {{ return x == 0 ? 32 : __builtin_clz((unsigned)x); }}
static int __clzll(long long x) {{ return x == 0 ? 64 : __builtin_clzll((unsigned long long)x); }}
{rule}
{caps}
int main(int argc, char **argv) {{
  if (argc > 1) {{  // tree_caps K: level count and capacities
    int cap[MAXLEV + 1];
    const int nl = tree_caps(atoi(argv[1]), cap);
    printf("%d", nl);
    for (int l = 0; l < nl; ++l) printf(" %d", cap[l]);
    printf("\\n");
    return 0;
  }}
  int m;
  if (scanf("%d", &m) != 1) return 1;
  std::vector<unsigned long long> key(m);
  std::vector<int> inst(m);
  for (int i = 0; i < m; ++i)
    if (scanf("%d %llx", &inst[i], &key[i]) != 2) return 1;
  // blocks of TPB elements staged with TG_H empty slots on each side, as tg_stage does
  for (int b0 = 0; b0 < m; b0 += TPB) {{
    uint64_t sk[TPB + 2 * TG_H];
    int32_t sq[TPB + 2 * TG_H];
    for (int t = 0; t < TPB + 2 * TG_H; ++t) {{
      const int i = b0 - TG_H + t;
      const bool v = i >= 0 && i < m;
      sk[t] = v ? key[i] : 0ull;
      sq[t] = v ? inst[i] : -1;
    }}
    for (int t = 0; t < TPB && b0 + t < m; ++t)
      if (tg_start(sk, sq, b0 + t, t)) printf("%d\\n", b0 + t);
  }}
  return 0;
}}
"""
    path = tmp_path / "tg.cpp"
    path.write_text(src)
    exe = tmp_path / "tg"
    subprocess.run([CXX, "-O2", "-std=c++17", "-o", str(exe), str(path)], check=True,
                   capture_output=True)
    return str(exe)


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    if CXX is None:
        pytest.skip("no C++ compiler")
    return _harness(tmp_path_factory.mktemp("tg"))


def _starts(exe, inst, key):
    inp = f"{len(key)}\n" + "".join(f"{int(q)} {int(k):x}\n" for q, k in zip(inst, key))
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
    return [int(x) for x in out.split()]


def _brute_starts(inst, key):
    """Largest cell of at most 32 elements containing each element: the
    elements sharing the most leading bits of (inst << 64 | key) with it,
    widened one bit at a time while the cell stays within 32."""
    full = [(int(q) << 64) | int(k) for q, k in zip(inst, key)]
    m = len(full)
    starts = set()
    i = 0
    while i < m:
        # the cell of prefix length l containing element i
        def cell(l):
            shift = 96 - l
            p = full[i] >> shift if shift < 96 else 0
            lo = i
            while lo > 0 and (full[lo - 1] >> shift if shift < 96 else 0) == p:
                lo -= 1
            hi = i + 1
            while hi < m and (full[hi] >> shift if shift < 96 else 0) == p:
                hi += 1
            return lo, hi
        lo, hi = None, None
        for l in range(0, 97):
            a, b = cell(l)
            if b - a <= 32:
                lo, hi = a, b
                break
        if lo is None:  # more than 32 equal keys: runs of 32 from the run's start
            a, b = cell(96)
            for s in range(a, b):
                if s == a or s % 32 == 0:
                    starts.add(s)
            i = b
            continue
        starts.add(lo)
        i = hi
    return sorted(starts)


def _keys(rng, m, ninst, dup_runs):
    inst = np.sort(rng.integers(0, ninst, size=m))
    key = np.zeros(m, dtype=np.uint64)
    for q in np.unique(inst):
        sel = np.flatnonzero(inst == q)
        centres = rng.integers(0, 2 ** 63, size=4, dtype=np.uint64)
        k = centres[rng.integers(0, 4, size=len(sel))] + rng.integers(
            0, 2 ** rng.integers(8, 40), size=len(sel), dtype=np.uint64)
        key[sel] = np.sort(k)
    for _ in range(dup_runs):  # runs of equal keys, some longer than 32
        a = int(rng.integers(0, m))
        ln = int(rng.integers(2, 80))
        b = min(m, a + ln)
        if np.all(inst[a:b] == inst[a]):
            key[a:b] = key[a]
    # keep each instance's keys sorted after planting the runs
    for q in np.unique(inst):
        sel = np.flatnonzero(inst == q)
        key[sel] = np.sort(key[sel])
    return inst, key


@pytest.mark.parametrize("seed", range(6))
def test_runs_are_the_largest_cells_of_at_most_32(harness, seed):
    rng = np.random.default_rng(seed)
    m = int(rng.integers(40, 1500))
    inst, key = _keys(rng, m, ninst=1 + seed % 3, dup_runs=seed)
    got = _starts(harness, inst, key)
    assert got == _brute_starts(inst, key)
    bounds = got + [m]
    assert all(0 < bounds[j + 1] - bounds[j] <= 32 for j in range(len(got)))


def test_small_levels_are_one_run(harness):
    for m in (1, 2, 17, 32):
        inst = np.zeros(m, dtype=np.int64)
        key = np.sort(np.random.default_rng(m).integers(0, 2 ** 60, size=m, dtype=np.uint64))
        assert _starts(harness, inst, key) == [0]


@pytest.mark.parametrize("K", [1, 2, 31, 32, 33, 248, 249, 2048, 4097, 10 ** 5, 10 ** 6,
                               10 ** 7, 2 ** 31 - 1])
def test_tree_caps(harness, K):
    out = subprocess.run([harness, str(K)], capture_output=True, text=True,
                         check=True).stdout.split()
    nl, cap = int(out[0]), [int(x) for x in out[1:]]
    assert len(cap) == nl and 1 <= nl <= 11
    assert cap[-1] <= 32                      # the top level fits one warp
    assert cap[0] >= -(-K // 32)              # fixed runs of 32 fit level 0
    for L in range(1, nl):                    # ... and every level above
        assert cap[L] >= -(-cap[L - 1] // 32)
    # the per-warp stack (STK = 288 in hac_query.cuh) holds 32 + 31 (levels - 1)
    stk = int(re.search(r"constexpr int STK = (\d+);",
                        open(os.path.join(CSRC, "hac_query.cuh")).read()).group(1))
    assert 32 + 31 * (nl - 1) <= stk
