import numpy as np


def rel_l2(a, b):
    """||a - b||_2 / ||b||_2 in FP64 (b is the FP64 oracle)."""
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


# FP32 tolerances the method is held to against the FP64 oracle.
TOL_CONV = 1e-5        # relative L2, one convolution
TOL_ITER = 1e-4        # relative L2 of x after up to 100 iterations
