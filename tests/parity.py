"""Comparison of a GPU decomposition with the FP64 oracle.

Integers (extrema counts, L, m, number of IMFs, stop reason) must be equal.
The only allowed differences are at an outer step where one side raised a
tie flag FOR THAT STEP: the GPU's per-IMF diagnostic record
(``diag[k].flags``) or the oracle's per-step record (``imf_flags[k]``).
EXTREMA_TIE (the oracle's MASK_TIE, same bit) excuses a different extrema
count or L at step k; NEAR_DELTA_TIE excuses a different m at IMF k.  There
the FP32 and FP64 paths may legitimately decide differently (several results
are correct).  The extrema count enters the method only through the stop
test (k < 2) and L: a flagged count difference that leaves both unchanged
(a count of thousands moves L = floor(nu n/k) only near an integer boundary)
is recorded and the comparison goes on; a difference in the stop decision, L
or m ends it at that step and is reported.  A flag raised at another IMF, or
either side's OR-ed status word, excuses nothing.  IMF relative L2 error must
stay below ``tol`` for every compared IMF and for the final remainder.
"""
from __future__ import annotations

import numpy as np

from paper_1802_01359_gb300 import fif

IMF_TOL = 1e-5


def rel_l2(a, b) -> float:
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def _np(a):
    return np.asarray(a.cpu().numpy() if hasattr(a, "cpu") else a)


def compare(got: fif.Decomposition, ref: dict, tol: float = IMF_TOL, signal=None) -> dict:
    """Returns a report dict; raises AssertionError on an unexcused mismatch.

    ``got`` must carry its per-IMF diagnostics (decompose with diag=True): they
    hold the GPU's flags per step and the extrema counts."""
    assert got.diag is not None, "parity.compare needs the GPU's per-IMF diag records"
    K_ref, K_got = ref["n_imfs"], got.n_imfs
    m, L = _np(got.m), _np(got.mask_len)
    imfs = _np(got.imfs).astype(np.float64)
    diag = got.diag
    rflags = ref["imf_flags"]
    rep = {"n_imfs": K_got, "errors": [], "diverged_at": None, "diverged_on": None,
           "count_ties": [], "flags": got.status & ~0xFF}
    for k in range(min(K_ref, K_got) + 1):
        gk = int(diag[k]["flags"])
        tie_ext = (gk | int(rflags[k])) & fif.FLAG_EXTREMA_TIE
        ke_g, ke_r = int(diag[k]["k_extrema"]), int(ref["kext"][k])
        if ke_g != ke_r:
            assert tie_ext, (
                f"extrema count differs at step {k}: gpu {ke_g} oracle {ke_r}, "
                "no EXTREMA_TIE at that step")
            rep["count_ties"].append(k)
            if (ke_g < 2) != (ke_r < 2):    # the stop test itself differs
                rep["diverged_at"], rep["diverged_on"] = k, "extrema"
                return rep
        if k == K_ref or k == K_got:
            break
        if L[k] != ref["L"][k]:
            assert tie_ext, f"L differs at IMF {k}: {L[k]} vs {ref['L'][k]}, no tie at that step"
            rep["diverged_at"], rep["diverged_on"] = k, "L"
            return rep
        if m[k] != ref["m"][k]:
            assert (gk | int(rflags[k])) & fif.FLAG_NEAR_DELTA_TIE, (
                f"m differs at IMF {k}: gpu {m[k]} oracle {ref['m'][k]} (L={L[k]}), "
                "no NEAR_DELTA_TIE at that IMF")
            rep["diverged_at"], rep["diverged_on"] = k, "m"
            return rep
        err = rel_l2(imfs[k], ref["imfs"][k])
        rep["errors"].append(err)
        assert err < tol, f"IMF {k} relative L2 error {err:.3e} >= {tol:g} (m={m[k]}, L={L[k]})"
    # equal extrema counts (and L) at every step give equal stop decisions
    assert K_got == K_ref, f"IMF count differs without a divergence: {K_got} vs {K_ref}"
    assert got.stop == ref["stop"], (got.status, ref["status"])
    rerr = rel_l2(imfs[K_got], ref["remainder"])
    rep["remainder_error"] = rerr
    assert rerr < tol, f"remainder relative L2 error {rerr:.3e}"
    return rep


def tie_fractions(statuses) -> dict:
    """Fraction of signals whose status word carries each tie flag."""
    st = np.asarray(statuses, dtype=np.int64)
    n = max(st.size, 1)
    return {"extrema_tie": float(((st & fif.FLAG_EXTREMA_TIE) != 0).sum() / n),
            "near_delta_tie": float(((st & fif.FLAG_NEAR_DELTA_TIE) != 0).sum() / n),
            "fp64_tiebreak": float(((st & fif.FLAG_FP64_TIEBREAK) != 0).sum() / n)}
