"""Error norms (Eq. 34 and companions)."""
import numpy as np


def l2_abs(a, b):
    """Eq. 34: sqrt(mean((a - b)^2)) over all nodes."""
    d = np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64)
    return float(np.sqrt(np.mean(d * d)))


def l2_rel(a, b):
    """||a - b||_2 / ||b||_2 (the parity measure)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (nb if nb > 0 else 1.0))


def linf(a, b):
    return float(np.max(np.abs(np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64))))
