"""Relative errors of the reconstructions (oracle), Eq. (RelativeError)."""
from __future__ import annotations

import numpy as np


def relative_error(true, rec) -> float:
    """E = 100 % ||true - rec|| / ||true|| (Euclidean norm over all cells)."""
    true = np.asarray(true, dtype=np.float64)
    rec = np.asarray(rec, dtype=np.float64)
    return 100.0 * float(np.linalg.norm(true - rec) / np.linalg.norm(true))
