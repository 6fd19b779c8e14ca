"""Modal reconstructor (FP64): Modalrec / Recmat (App. A, Tabs. 3-4; App. B,
Listing 2 ``recmat_object``): modes = R @ slopes, R of shape
(n_modes, n_slopes), slopes in the all-x-then-all-y layout."""
import numpy as np


def mvm(R: np.ndarray, s: np.ndarray) -> np.ndarray:
    """m = R s for one slope vector (n_slopes,) or a batch (n_batch, n_slopes)."""
    R = np.asarray(R, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    if s.ndim == 1:
        return R @ s
    return s @ R.T
