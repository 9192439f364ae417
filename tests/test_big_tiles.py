"""The GPU-wide pair evaluation's tile plan on the CPU: for every request a
batch can hold (larger side nL, smaller side nS, nL + nS <= n, any d and
kind), the tiles the scheduler gives it fit in the per-request share of the
partials buffer the library allocates, max(BIG_MAXT, ceil(n / BIG_TILE) + 1),
and the chunks cover the smaller cluster.  Compiled from the library's own
tile-shape functions; no CUDA call runs."""
import os
import subprocess

import pytest

from paper_2106_04727_gb300 import build

PROG = r"""
#include "hac_impl.cuh"
#include <cstdio>
#include <random>

using namespace hacg;

static long long per_request(long long n) {
  return std::max<long long>(BIG_MAXT, (n + BIG_TILE - 1) / BIG_TILE + 1);
}

static int check(long long n, int nL, int nS, int d, bool exact) {
  const int kind = bk_kind(nL, exact, d);
  const int w = bk_width(kind, d), c = bk_chunk(kind, nL, nS, d);
  const long long tl = (nL + w - 1) / w, ts = (nS + c - 1) / c;
  const long long tiles = tl * ts;
  if (c < 1 || ts * c < nS || tl * w < nL || tiles > per_request(n) || tiles > 0x7fffffff) {
    printf("n %lld nL %d nS %d d %d exact %d: kind %d width %d chunk %d tiles %lld > %lld\n",
           n, nL, nS, d, (int)exact, kind, w, c, tiles, per_request(n));
    return 1;
  }
  return 0;
}

int main() {
  std::mt19937_64 rng(11);
  long long cases = 0;
  const long long ns[] = {2, 3, 513, 2049, 4096, 65536, 1000000, 10000000, 100000000,
                          1073741823};
  for (long long n : ns)
    for (int d = 1; d <= 16; ++d)
      for (int ex = 0; ex < 2; ++ex) {
        // edges: the most lopsided and the most even splits
        const long long lo = 1, hi = n - 1;
        const long long edge[][2] = {{hi, lo}, {(n + 1) / 2, n / 2}, {n / 2, n / 2}};
        for (auto &e : edge) {
          if (e[1] < 1 || e[0] < e[1] || e[0] + e[1] > n) continue;
          if (check(n, (int)e[0], (int)e[1], d, ex)) return 1;
          ++cases;
        }
        for (int k = 0; k < 2000; ++k) {
          const long long nL = 1 + (long long)(rng() % (unsigned long long)(n - 1));
          const long long room = std::min(nL, n - nL);
          if (room < 1) continue;
          const long long nS = 1 + (long long)(rng() % (unsigned long long)room);
          if (check(n, (int)nL, (int)nS, d, ex)) return 1;
          ++cases;
        }
      }
  printf("ok %lld\n", cases);
  return 0;
}
"""


def test_tile_plan_fits_the_partials_buffer(tmp_path):
    try:
        nv = build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not found")
    src = tmp_path / "tiles.cu"
    src.write_text(PROG)
    exe = tmp_path / "tiles"
    r = subprocess.run([nv, *build._flags(), str(src), "-o", str(exe)], capture_output=True,
                       text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout[-1000:]
    ok, cases = out.stdout.split()
    assert ok == "ok" and int(cases) > 500000
