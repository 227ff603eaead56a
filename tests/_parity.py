"""Shared helpers of the GPU parity tests (comparison metrics only)."""
import numpy as np

# Receiver and volume Green's functions: relative L2 error over the entries
# whose magnitude exceeds 1e-6 of the largest one, per field kind (E or H,
# which carry different units).  2e-4 is the bound the FP32 path must meet
# against the FP64 oracle.
REL_L2_TOL = 2e-4
MASK_FLOOR = 1e-6


def rel_l2_masked(got, ref, floor=MASK_FLOOR):
    got = np.asarray(got).ravel()
    ref = np.asarray(ref).ravel()
    keep = np.abs(ref) > floor * np.abs(ref).max()
    if not keep.any():
        return 0.0
    return float(np.linalg.norm(got[keep] - ref[keep]) / np.linalg.norm(ref[keep]))


def max_rel_masked(got, ref, floor=MASK_FLOOR):
    got = np.asarray(got).ravel()
    ref = np.asarray(ref).ravel()
    keep = np.abs(ref) > floor * np.abs(ref).max()
    return float(np.max(np.abs(got[keep] - ref[keep]) / np.abs(ref[keep]))) if keep.any() else 0.0


def compare_G(got, ref):
    """(rel_l2_E, rel_l2_H) for receiver arrays [nrec, 6, nfreq] or volume
    arrays [6, nfreq, ...]."""
    got, ref = np.asarray(got), np.asarray(ref)
    if got.ndim == 3 and got.shape[1] == 6:
        return rel_l2_masked(got[:, :3], ref[:, :3]), rel_l2_masked(got[:, 3:], ref[:, 3:])
    return rel_l2_masked(got[:3], ref[:3]), rel_l2_masked(got[3:], ref[3:])
