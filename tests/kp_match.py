"""Keypoint-set comparison used by the parity tests.

Two keypoints match when they sit on the same level within 0.5 px.  A
keypoint present on one side only is an expected miss when the decision that
admits it is within floating-point reach of its boundary on the oracle's
FP64 response: the response within `tol` of the threshold or of its largest
26-neighbour, the edge ratio within 1e-3 of (r+1)^2/r, or a sub-pixel offset
within 1e-3 of one pixel.  Overlap = matched / max(|A|, |B|) after the
expected misses are removed from both sides.
"""
import numpy as np


def _decision_margin_ok(D, lvl, y, x, thr, edge_r, tol):
    """True if the oracle response at (lvl, y, x) is near a decision boundary."""
    n, h, w = D.shape
    if not (1 <= lvl <= n - 2 and 1 <= y <= h - 2 and 1 <= x <= w - 2):
        return False
    v = D[lvl, y, x]
    if abs(v - thr) <= tol:
        return True
    cube = D[lvl - 1:lvl + 2, y - 1:y + 2, x - 1:x + 2].copy()
    cube[1, 1, 1] = -np.inf
    if abs(v - cube.max()) <= tol:
        return True
    P = D[lvl, y - 1:y + 2, x - 1:x + 2]
    gx = 0.5 * (P[1, 2] - P[1, 0])
    gy = 0.5 * (P[2, 1] - P[0, 1])
    hxx = P[1, 2] - 2 * P[1, 1] + P[1, 0]
    hyy = P[2, 1] - 2 * P[1, 1] + P[0, 1]
    hxy = 0.25 * (P[2, 2] - P[2, 0] - P[0, 2] + P[0, 0])
    det = hxx * hyy - hxy * hxy
    tr = hxx + hyy
    if edge_r > 0:
        lim = (edge_r + 1) ** 2 / edge_r
        if det != 0 and abs(tr * tr / det - lim) <= 1e-3 * lim:
            return True
        if abs(det) <= 1e-6 * (hxx * hxx + hyy * hyy + 1e-300):
            return True
    if det != 0:
        ox = -(hyy * gx - hxy * gy) / det
        oy = -(hxx * gy - hxy * gx) / det
        if abs(abs(ox) - 1) <= 1e-3 or abs(abs(oy) - 1) <= 1e-3:
            return True
    return False


def compare(kp_ref, kp_got, D_ref, thr=0.001, edge_r=10.0, rel_tol=1e-4, dist=0.5):
    """Returns (overlap, n_matched, unexplained_ref, unexplained_got, max_dist)."""
    tol_lvl = rel_tol * np.max(np.abs(D_ref.reshape(D_ref.shape[0], -1)), axis=1)
    used = np.zeros(len(kp_got), dtype=bool)
    by_level = {}
    for j, k in enumerate(kp_got):
        by_level.setdefault(int(k["level"]), []).append(j)
    matched = 0
    max_d = 0.0
    miss_ref = []
    for k in kp_ref:
        best, bd = -1, dist
        for j in by_level.get(int(k["level"]), []):
            if used[j]:
                continue
            d = float(np.hypot(float(kp_got[j]["x"]) - k["x"], float(kp_got[j]["y"]) - k["y"]))
            if d <= bd:
                best, bd = j, d
        if best >= 0:
            used[best] = True
            matched += 1
            max_d = max(max_d, bd)
        else:
            miss_ref.append(k)
    miss_got = [kp_got[j] for j in range(len(kp_got)) if not used[j]]

    def unexplained(miss):
        out = []
        for k in miss:
            lvl, y, x = int(k["level"]), int(k["iy"]), int(k["ix"])
            if not _decision_margin_ok(D_ref, lvl, y, x, thr, edge_r, tol_lvl[lvl]):
                out.append(k)
        return out

    ur = unexplained(miss_ref)
    ug = unexplained(miss_got)
    n_ref = len(kp_ref) - (len(miss_ref) - len(ur))
    n_got = len(kp_got) - (len(miss_got) - len(ug))
    denom = max(n_ref, n_got)
    overlap = 1.0 if denom == 0 else matched / denom
    return overlap, matched, ur, ug, max_d
