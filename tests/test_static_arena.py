"""The allocation-free entry point's memory plan on the CPU: for every
dimension, input type and linkage, the arrays of an n = HAC_STATIC_MAX_N
instance are carved from the fixed device array without running past it, as
the library's own carving code lays them out (compiled from its source; no
CUDA call runs)."""
import glob
import os
import subprocess

import pytest

from paper_2106_04727_gb300 import build

PROG = r"""
#include "hac_core.cu"
#include <cstdio>

int main() {
  size_t most = 0;
  for (int lk = 0; lk < 4; ++lk)
    for (int dt = 0; dt < 2; ++dt)
      for (int d = 1; d <= MAXD; ++d) {
        hac_ctx h;
        h.n = HAC_STATIC_MAX_N;
        h.d = d;
        h.dt = (hac_dtype)dt;
        h.lk = (hac_linkage)lk;
        h.s.n = h.n;
        h.s.d = d;
        h.s.dp = pad_dim(d);
        h.s.linkage = lk;
        // offsets only: the base stands for the array's (256-byte aligned) address
        Carver cv{(unsigned char *)nullptr + 256, 0, kStaticArenaBytes, true};
        if (!carve_state(h, cv) || cv.off > kStaticArenaBytes) {
          printf("lk %d dt %d d %d: %zu bytes of %zu\n", lk, dt, d, cv.off, kStaticArenaBytes);
          return 1;
        }
        most = cv.off > most ? cv.off : most;
      }
  printf("ok %zu %zu\n", most, kStaticArenaBytes);
  return 0;
}
"""


def test_static_arena_holds_the_largest_instance(tmp_path):
    try:
        nv = build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not found")
    build.build()
    objs = [o for o in glob.glob(os.path.join(build.BUILD, "*.o"))
            if os.path.basename(o) != "hac_core.o"]
    src = tmp_path / "arena.cu"
    src.write_text(PROG)
    exe = tmp_path / "arena"
    r = subprocess.run([nv, *build._flags(), str(src), *objs, "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout[-1000:]
    ok, most, cap = out.stdout.split()
    assert ok == "ok" and 0 < int(most) <= int(cap)
