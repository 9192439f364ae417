"""hac_run_static: the clustering entry point that allocates nothing.

It serves callers that cannot call cudaMalloc when they need a dendrogram
(a memory pool that already owns the whole GPU, or latency-sensitive code that
must not risk the device-wide synchronisation cudaMalloc/cudaFree can cause).
Its working memory is a fixed array inside the library, so its output must be
the same as the ordinary create/run/dendrogram path's, call after call, even
though every call reuses (and overwrites) that array.

This file is collected last on purpose: a failure here should not stop the
rest of the suite from running first.
"""
import numpy as np
import pytest

import oracle
from paper_2106_04727_gb300 import hac, inputs


def test_static_rejects_sizes_beyond_its_maximum():
    """The size check runs before any CUDA call (no GPU needed)."""
    lib = hac.load()
    n = hac.HAC_STATIC_MAX_N + 1
    rc = lib.hac_run_static(1, n, 2, hac.F32, hac.WARD, None, 1, n - 1)
    assert rc == hac.HAC_EINVAL
    rc = lib.hac_run_static(1, 10, 2, hac.F32, hac.WARD, None, 1, 5)
    assert rc == hac.HAC_ECAP


def _static(torch, X, lk, prec, bufs):
    """One hac_run_static call on preallocated device buffers (points, and
    n - 1 records of 32 bytes)."""
    n, d = X.shape
    src, out = bufs
    rc = hac.hac_run_static(src.data_ptr(), n, d, X.dtype, lk, out.data_ptr(), n - 1,
                            precision=prec)
    assert rc == hac.HAC_OK, hac.hac_strerror(rc)
    rec = out.cpu().numpy().view(hac.MERGE_DTYPE)
    return dict(a=rec["cid_a"], b=rec["cid_b"], h=rec["height"], size=rec["size"])


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [hac.PREC_F64, hac.PREC_F32_RECHECK], ids=["f64", "f32recheck"])
def test_static_matches_allocating_path_twice(prec, monkeypatch):
    """Same dendrogram as the allocating path (which, like this entry point,
    stays on the range-query search here: no dense matrix) and as the CPU
    oracle, on consecutive calls that reuse (and overwrite) the fixed array,
    and no device memory taken by those calls."""
    torch = pytest.importorskip("torch")
    monkeypatch.setenv("HAC_DENSE_K", "0")
    cases = [(inputs.gaussian_mixture(3000, 5, 12, seed=91), "ward"),
             (inputs.uniform_cube(hac.HAC_STATIC_MAX_N, 2, seed=92, dtype=np.float64), "average"),
             (inputs.gaussian_mixture(777, 3, 4, seed=93), "complete")]
    # everything that allocates runs before the measured region: the
    # allocating path, the oracle, and the device buffers of every call
    wants = [hac.cluster(X, lk, precision=prec, with_rounds=False) for X, lk in cases]
    refs = [oracle.nnchain(X.astype(np.float64), lk) for X, lk in cases]
    bufs = [(torch.from_numpy(X).cuda(),
             torch.zeros((len(X) - 1) * 4, dtype=torch.int64, device="cuda")) for X, _ in cases]
    torch.cuda.synchronize()
    _static(torch, *cases[0], prec, bufs[0])   # loads the library's module on this device
    free0 = torch.cuda.mem_get_info()[0]
    for i in (0, 1, 2, 0):                     # consecutive calls reuse the same array
        X, lk = cases[i]
        got = _static(torch, X, lk, prec, bufs[i])
        c = oracle.compare(got, wants[i], rtol=1e-9)
        assert c["ok"], (lk, c)
        # same canonical order as hac_dendrogram
        assert np.array_equal(got["a"], wants[i]["a"]) and np.array_equal(got["b"], wants[i]["b"])
        # FP32 mode: complete / average heights carry the stated FP32 bound
        rtol = 1e-5 if prec == hac.PREC_F32_RECHECK and lk in ("complete", "average") else 1e-9
        c = oracle.compare(got, refs[i], rtol=rtol)
        assert c["ok"], (lk, "oracle", c)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
