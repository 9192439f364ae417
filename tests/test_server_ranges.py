"""The serving engines' free-range allocator on the CPU: first fit over the
free cid ranges and coalescing on release, checked step by step against a
bitmap model by a small host program compiled from the server's own source
(no CUDA call runs)."""
import glob
import os
import subprocess

import pytest

from paper_2106_04727_gb300 import build

PROG = r"""
#include "hac_server.cu"
#include <cstdio>
#include <random>

int main() {
  const int N = 4096;
  Engine e;
  e.free_ranges = {{0, N}};
  std::vector<char> used(N, 0), fr(N, 0);
  std::vector<std::pair<int, int>> held;
  std::mt19937 rng(7);
  long takes = 0, refusals = 0, gives = 0;
  for (int step = 0; step < 100000; ++step) {
    const bool take = held.empty() || rng() % 100 < 55;
    if (take) {
      const int n = 1 + (int)(rng() % (rng() % 4 == 0 ? 700 : 40));
      int want = -1;  // model: start of the first free run of at least n cells
      for (int i = 0, run = 0; i < N; ++i) {
        run = used[i] ? 0 : run + 1;
        if (run == n) {
          want = i - n + 1;
          break;
        }
      }
      int base = -1;
      const bool ok = range_take(e, n, &base);
      if (ok != (want >= 0) || (ok && base != want)) {
        printf("step %d take %d: got %d at %d, model %d\n", step, n, (int)ok, base, want);
        return 1;
      }
      if (ok) {
        for (int i = base; i < base + n; ++i) used[i] = 1;
        held.push_back({base, n});
        ++takes;
      } else {
        ++refusals;
      }
    } else {
      const size_t k = rng() % held.size();
      const auto r = held[k];
      held.erase(held.begin() + k);
      range_give(e, r.first, r.second);
      for (int i = r.first; i < r.first + r.second; ++i) used[i] = 0;
      ++gives;
    }
    // the ranges are sorted, non-empty, neither overlapping nor touching
    // (touching ones must have been coalesced), and cover the free cells
    std::fill(fr.begin(), fr.end(), 0);
    int prev_end = -1;
    for (const auto &r : e.free_ranges) {
      if (r.second <= 0 || r.first <= prev_end || r.first + r.second > N) {
        printf("step %d: bad range (%d, %d) after end %d\n", step, r.first, r.second, prev_end);
        return 2;
      }
      for (int i = r.first; i < r.first + r.second; ++i) fr[i] = 1;
      prev_end = r.first + r.second;
    }
    for (int i = 0; i < N; ++i)
      if (fr[i] == used[i]) {
        printf("step %d: cell %d free in ranges %d, used in model %d\n", step, i, fr[i], used[i]);
        return 3;
      }
  }
  printf("ok %ld %ld %ld\n", takes, refusals, gives);
  return 0;
}
"""


def test_free_range_allocator_matches_bitmap_model(tmp_path):
    try:
        nv = build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not found")
    build.build()
    objs = [o for o in glob.glob(os.path.join(build.BUILD, "*.o"))
            if os.path.basename(o) != "hac_server.o"]
    src = tmp_path / "ranges.cu"
    src.write_text(PROG)
    exe = tmp_path / "ranges"
    r = subprocess.run([nv, *build._flags(), str(src), *objs, "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout[-1000:]
    ok, takes, refusals, gives = out.stdout.split()
    assert ok == "ok" and int(takes) > 10000 and int(refusals) > 100 and int(gives) > 10000
