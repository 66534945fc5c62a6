"""The error-rate protocol used by the sweep workload (the paper's accuracy
table): checked on hand-made arrays whose answer is known."""
import numpy as np

import bench


def test_accuracy_counts():
    H, W = 4, 5
    gt = np.full((H, W), 10.0, np.float32)
    occ = np.zeros((H, W), bool)
    occ[0, 0] = True                       # occluded: not counted
    mask = np.ones((H, W), np.uint8)
    mask[3, :] = 0                         # outside Omega_I: not counted
    D = gt.copy()
    D[1, 0] = 12.5                         # 2.5 px off
    D[1, 1] = 14.5                         # 4.5 px off
    C = np.zeros((H, W), np.uint8)
    C[2, 0] = 8                            # not validated (C_f == t_hi): outside the error rates
    r = bench.accuracy(D, C, mask, gt, occ, t_hi=8)
    n = 3 * 5 - 1                          # Omega_I rows 0..2, minus the occluded pixel
    nv = n - 1                             # minus the unvalidated pixel
    assert r["density"] == nv / n
    assert r["lt2px"] == (nv - 2) / nv
    assert r["lt3px"] == (nv - 1) / nv
    assert r["lt4px"] == (nv - 1) / nv
    assert r["lt5px"] == nv / nv
