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


def j2_point_errors(state, stress, ref_state, ref_stress, mask, young=1.0, poisson=0.3):
    """Per-point normwise errors of the J2 update against the oracle.

    The scale of a point is the size of the strain that drives its update,
    S = max|eps_p| + |alpha| + max|sigma| / (2 mu), from the oracle's state
    and stress.  The return map is FP64 on both sides, so rounding moves the
    state by about 1e-16 S; a tie in Newton's stopping test moves dgamma by at
    most tol_g sigma_y / |g'| (about 1e-13 S at the default tolerances), and a
    tie in the yield decision (f_trial within rounding of 0) by as little.
    Returns (max over points of |state - ref| / S, of |stress - ref| /
    ((3 kappa + 2 mu) S)); a point with S == 0 must match exactly.
    ``stress`` may be None (the assembly keeps no stress).
    """
    mu = young / (2.0 * (1.0 + poisson))
    kappa = young / (3.0 * (1.0 - 2.0 * poisson))
    rs, rsig = np.asarray(ref_state)[mask], np.asarray(ref_stress)[mask]
    S = np.abs(rs[:, :6]).max(axis=1) + np.abs(rs[:, 6]) + np.abs(rsig).max(axis=1) / (2.0 * mu)
    ds = np.abs(np.asarray(state)[mask] - rs).max(axis=1)
    zero = S == 0
    assert np.all(ds[zero] == 0), "a point with no strain has a state"
    err_state = float(np.max(ds[~zero] / S[~zero])) if (~zero).any() else 0.0
    err_stress = 0.0
    if stress is not None:
        dsig = np.abs(np.asarray(stress)[mask] - rsig).max(axis=1)
        assert np.all(dsig[zero] == 0), "a point with no strain has a stress"
        if (~zero).any():
            err_stress = float(np.max(dsig[~zero] / ((3.0 * kappa + 2.0 * mu) * S[~zero])))
    return err_state, err_stress
