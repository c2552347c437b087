"""Shared helpers of the test-suite: engine loading, oracle comparisons."""
import numpy as np
import pytest

FP64_TOL = 1e-12   # max |a - r| / S for the FP64 path
FP32_TOL = 1e-5    # same metric, FP32-integrate / FP64-accumulate path


def engine():
    """The CUDA engine binding; builds the library if needed (GPU tests only)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_03949_gb300 import build
    build.build()
    from paper_1805_03949_gb300 import fea
    return fea


def err_vs_oracle(a, ref, S):
    """max |a - ref| / S over S > 0, and max |a| / max(S) over S == 0.

    S is the oracle's normwise scale of each entry (the Cauchy-Schwarz bound of
    its quadrature terms, ``NA``/``Nb``): rounding the gradients by a relative
    eps moves an entry by about eps * S, whatever cancellation the entry has.
    Entries with S == 0 (no gradient at all) must stay at rounding level of
    the largest S.
    """
    a = np.asarray(a); ref = np.asarray(ref); S = np.asarray(S)
    pos = S > 0
    err = float(np.max(np.abs(a[pos] - ref[pos]) / S[pos])) if pos.any() else 0.0
    smax = float(S.max()) if S.size else 0.0
    zero_dev = float(np.max(np.abs(a[~pos]))) / smax if ((~pos).any() and smax > 0) else 0.0
    return err, zero_dev
