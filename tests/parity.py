"""Comparison of a GPU decomposition with the FP64 oracle.

Integers (extrema counts, L, m, number of IMFs, stop reason) must be equal.
The only allowed divergence is at an outer step where the GPU itself raised a
tie flag (NEAR_DELTA_TIE for m, EXTREMA_TIE for the extrema count): there the
FP32 and FP64 paths may legitimately decide differently, and the comparison
stops at that step and reports it.  IMF relative L2 error must stay below
``tol`` for every compared IMF and for the final remainder.
"""
from __future__ import annotations

import numpy as np

from paper_1802_01359_gb300 import fif

IMF_TOL = 1e-5


def rel_l2(a, b) -> float:
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def compare(got: fif.Decomposition, ref: dict, tol: float = IMF_TOL, signal=None) -> dict:
    """Returns a report dict; raises AssertionError on an unflagged mismatch."""
    K_ref, K_got = ref["n_imfs"], got.n_imfs
    m = np.asarray(got.m.cpu().numpy() if hasattr(got.m, "cpu") else got.m)
    L = np.asarray(got.mask_len.cpu().numpy() if hasattr(got.mask_len, "cpu") else got.mask_len)
    imfs = got.imfs.cpu().numpy() if hasattr(got.imfs, "cpu") else np.asarray(got.imfs)
    imfs = imfs.astype(np.float64)
    diag = got.diag
    rep = {"n_imfs": K_got, "errors": [], "diverged_at": None, "flags": got.status & ~0xFF}
    for k in range(max(K_ref, K_got) + 1):
        kflags = int(diag[k]["flags"]) if diag is not None and k < len(diag) else got.status
        if diag is not None and k <= min(K_ref, K_got):
            if int(diag[k]["k_extrema"]) != int(ref["kext"][k]):
                assert kflags & fif.FLAG_EXTREMA_TIE, (
                    f"extrema count differs at step {k}: gpu {int(diag[k]['k_extrema'])} "
                    f"oracle {int(ref['kext'][k])}, no EXTREMA_TIE flag")
                rep["diverged_at"] = k
                return rep
        if k >= K_ref or k >= K_got:
            break
        if L[k] != ref["L"][k]:
            assert kflags & fif.FLAG_EXTREMA_TIE, f"L differs at IMF {k}: {L[k]} vs {ref['L'][k]}"
            rep["diverged_at"] = k
            return rep
        if m[k] != ref["m"][k]:
            assert kflags & fif.FLAG_NEAR_DELTA_TIE or ref["status"] & fif.FLAG_NEAR_DELTA_TIE, (
                f"m differs at IMF {k}: gpu {m[k]} oracle {ref['m'][k]} (L={L[k]}), no tie flag")
            rep["diverged_at"] = k
            return rep
        err = rel_l2(imfs[k], ref["imfs"][k])
        rep["errors"].append(err)
        assert err < tol, f"IMF {k} relative L2 error {err:.3e} >= {tol:g} (m={m[k]}, L={L[k]})"
    if K_got != K_ref:
        assert got.status & fif.FLAG_EXTREMA_TIE, f"IMF count differs: {K_got} vs {K_ref}"
        rep["diverged_at"] = min(K_got, K_ref)
        return rep
    assert got.stop == ref["stop"], (got.status, ref["status"])
    rerr = rel_l2(imfs[K_got], ref["remainder"])
    rep["remainder_error"] = rerr
    assert rerr < tol, f"remainder relative L2 error {rerr:.3e}"
    return rep
