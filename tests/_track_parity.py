"""Tracking parity rule shared by the GPU tests: one frame pair of the CUDA path's
corner selection and Lucas-Kanade step against the FP64 oracle.

The CUDA path ranks corners by its FP32 response, the oracle by FP64: the selected sets
agree except for corners whose oracle response is within the FP32 tolerance of the K-th
response; velocities of the common points agree within 2e-3 px/frame, scaled by the
window's conditioning; status flags agree away from the singularity threshold.
"""
from __future__ import annotations

import numpy as np

from oracle import chain as oc
from tests._parity import TOL_F32, exempt_pixels


def window_conditioning(maps_cur, g_prev, p, W, H):
    """|det| / tr^2 of the oracle's LK matrix at raster index p (for the tolerance only)."""
    py, px = divmod(int(p), W)
    ys = np.clip(np.arange(py - 3, py + 4), 0, H - 1)
    xs = np.clip(np.arange(px - 3, px + 4), 0, W - 1)
    gx = maps_cur["ix"][np.ix_(ys, xs)] / 8
    gy = maps_cur["iy"][np.ix_(ys, xs)] / 8
    a00, a01, a11 = np.sum(gx * gx), np.sum(gx * gy), np.sum(gy * gy)
    det, tr = a00 * a11 - a01 * a01, a00 + a11
    return abs(det) / (tr * tr) if tr > 0 else 0.0


def check_frame(fr, t, W, out, Kp, tol=TOL_F32, exempt_corners=False):
    """One frame pair. With exempt_corners, a point may also differ where the corner
    decision itself is exempt under the mask rule (its response within tol * max|R| of
    the threshold or of a neighbour's): a lower precision may flip such a decision at any
    strength, not only at the K-th response."""
    H = fr.shape[1]
    prev, cur = fr[t - 1][:, :W].copy(), fr[t][:, :W].copy()
    idx_o, u_o, v_o, st_o = oc.track_pair(prev, cur, K=Kp)
    maps, mask_o, _ = oc.chain_frame(cur)
    n = int(out["n"][t])
    assert n == len(idx_o)
    got = out["idx"][t, :n]
    r = maps["r"].ravel()
    if n:
        tau = tol * np.max(np.abs(maps["r"]))
        kth = r[idx_o[-1]]
        diff = set(got.tolist()) ^ set(idx_o.tolist())
        ex = exempt_pixels(maps["r"], tol).ravel() if exempt_corners else None
        for p in diff:  # disagreements only at the selection boundary (or exempt decisions)
            assert abs(r[p] - kth) <= tau or (ex is not None and ex[p]), (t, p, r[p], kth)
        # order: strongest first (by the oracle's response, up to the FP32 tolerance)
        assert np.all(np.diff(r[got]) <= tau)
    g_prev = oc.chain_frame(prev)[0]["g"]
    common = {p: i for i, p in enumerate(idx_o.tolist())}
    checked = 0
    for i, p in enumerate(got.tolist()):
        if p not in common:
            continue
        j = common[p]
        cond = window_conditioning(maps, g_prev, p, W, H)
        if cond < 1e-9 or (1e-13 < cond < 1e-11):
            continue  # at or near the singularity threshold: either answer is acceptable
        assert out["st"][t, i] == st_o[j], (t, p)
        if st_o[j] == 0:
            vtol = 2e-3 * max(1.0, 1e-4 / cond)  # FP32 window sums, amplified by conditioning
            assert abs(out["u"][t, i] - u_o[j]) <= vtol * max(1.0, abs(u_o[j])), (t, p, out["u"][t, i], u_o[j])
            assert abs(out["v"][t, i] - v_o[j]) <= vtol * max(1.0, abs(v_o[j])), (t, p, out["v"][t, i], v_o[j])
            checked += 1
    return checked
