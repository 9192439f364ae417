"""Host logic of the threshold tuner, on the CPU: every combination of the
grid is run with its environment set before the handle is created, and the
fastest median is reported (the library calls are replaced by fakes here)."""
import json

from paper_2106_04727_gb300 import hac, inputs, tune


def test_grid_environment_and_best(monkeypatch, capsys):
    seen = []
    fake_ms = {(32768, 131072): 9.0, (32768, 262144): 7.0, (65536, 131072): 5.0,
               (65536, 262144): 6.0}

    class H:
        def __init__(self, key):
            self.key = key

    def create(X, linkage):
        import os
        key = (int(os.environ["HAC_BIG_PAIRS"]), int(os.environ["HAC_WARP_BUDGET"]))
        seen.append((key, linkage, len(X)))
        return H(key)

    runs = []

    def run(h, precision, cache_slots):
        runs.append((h.key, precision, cache_slots))
        return hac.HAC_OK

    def stats(h):
        return {"ms_total": fake_ms[h.key], "point_pairs": 1, "ms_query": 0.5, "ms_big": 0.25}

    monkeypatch.setattr(hac, "hac_create", create)
    monkeypatch.setattr(hac, "hac_run", run)
    monkeypatch.setattr(hac, "hac_stats", stats)
    monkeypatch.setattr(hac, "hac_destroy", lambda h: None)
    monkeypatch.setattr(inputs, "workload", lambda name, n=None: [[0.0, 0.0]] * (n or 7))
    # the tuner sets these for the library; restore them after the test
    monkeypatch.setenv("HAC_BIG_PAIRS", "0")
    monkeypatch.setenv("HAC_WARP_BUDGET", "0")
    tune.main(["--big", "32768,65536", "--budget", "131072,262144", "--slots", "64",
               "--runs", "2", "--n", "5", "--linkage", "complete"])
    lines = [json.loads(x) for x in capsys.readouterr().out.splitlines()]
    assert len(lines) == 5
    assert sorted(k for k, _, _ in seen) == sorted(fake_ms)
    assert all(lk == "complete" and n == 5 for _, lk, n in seen)
    # one warm-up and two timed runs per combination, FP32 + re-score, the slots asked for
    assert len(runs) == 12 and all(p == hac.PREC_F32_RECHECK and s == 64 for _, p, s in runs)
    best = lines[-1]["best"]
    assert (best["HAC_BIG_PAIRS"], best["HAC_WARP_BUDGET"]) == (65536, 131072)
    assert best["ms"] == 5.0 and lines[-1]["n"] == 5


def test_shape_grid_builds_and_times_each_variant(monkeypatch, capsys):
    """--shapes: one compiled variant per combination of the macro values,
    each timed in a child process; the fastest is reported."""
    import subprocess
    import sys

    from paper_2106_04727_gb300 import build

    assert tune.shape_grid("HAC_DS_PPT8=2,4;HAC_QWARPS=4") == [
        {"HAC_DS_PPT8": 2, "HAC_QWARPS": 4}, {"HAC_DS_PPT8": 4, "HAC_QWARPS": 4}]
    try:
        tune.shape_grid("HAC_NOT_A_SHAPE=1")
        raise AssertionError("an unknown macro must be refused")
    except ValueError:
        pass
    built, cmds = [], []
    monkeypatch.setattr(build, "build", lambda defines=None, **k: built.append(defines) or
                        f"/v/{defines['HAC_DS_MINB']}/libhac.so")
    ms = {"/v/2/libhac.so": 8.0, "/v/3/libhac.so": 6.5}

    def run(cmd, capture_output, text):
        cmds.append(cmd)
        lib = cmd[cmd.index("--lib") + 1]
        out = json.dumps({"best": {"ms": ms[lib], "ms_search": 1.0}})
        return subprocess.CompletedProcess(cmd, 0, stdout=out + "\n", stderr="")

    monkeypatch.setattr(subprocess, "run", run)
    tune.main(["--shapes", "HAC_DS_MINB=2,3", "--workload", "gmm5d_1m_f32", "--n", "9"])
    lines = [json.loads(x) for x in capsys.readouterr().out.splitlines()]
    assert built == [{"HAC_DS_MINB": 2}, {"HAC_DS_MINB": 3}]
    assert all(c[0] == sys.executable and "--lib" in c and c[c.index("--n") + 1] == "9"
               for c in cmds)
    assert lines[-1]["best"] == {"HAC_DS_MINB": 3, "ms": 6.5, "ms_search": 1.0}
