"""Error norm of the oracle (test infrastructure).

Eq. 10 (Sec. 2.3.3): L2(phi) = sqrt(sum_i |phi_i^a - phi_i^n|^2) / sqrt(sum_i |phi_i^a|^2),
where phi^a is the reference ("analytical") value and phi^n the approximation;
for vector fields |.| is the Euclidean norm of the per-particle vector.
"""
import numpy as np


def l2_error(reference, approx):
    ref = np.asarray(reference, dtype=np.float64)
    app = np.asarray(approx, dtype=np.float64)
    num = np.sqrt(np.sum((ref - app) ** 2))
    den = np.sqrt(np.sum(ref ** 2))
    return float(num / den)
