"""Tolerances shared by the GPU tests, derived from the arithmetic."""
import numpy as np

FP32_U = 6e-8  # FP32 unit roundoff (2^-24)


def descriptor_tol(G, m):
    """Bound on the FP32 rounding error of every descriptor coefficient.

    Each coefficient is an FP32 sum of terms with |T_a| <= 1, so its error is a
    small multiple of u times the sum of |terms|, which is at most max|s|^p * G_0
    of its block (G_0 = the a = 0 coefficient; p = 0 unweighted, 1 weighted
    radial, 2 weighted angular). Allowed: 32 u times that bound, plus 1e-6."""
    Kr, Ka = m.order_rad + 1, m.order_ang + 1
    smax = float(np.abs(m.type_weights).max())
    B = np.empty_like(G)
    B[:, :Kr] = G[:, [0]]
    B[:, Kr:Kr + Ka] = G[:, [Kr]]
    B[:, Kr + Ka:2 * Kr + Ka] = smax * G[:, [0]]
    B[:, 2 * Kr + Ka:] = smax ** 2 * G[:, [Kr]]
    return 32 * FP32_U * np.abs(B) + 1e-6
