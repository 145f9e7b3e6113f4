"""Error metrics shared by the parity tests (relative L2 per conserved field)."""
import numpy as np


def field_errors(q, ref):
    """Relative L2 errors of a (5, ...) state against a reference:
    rho and E against their own norms, the momentum as one vector field
    (near-zero components carry no norm of their own)."""
    q = np.asarray(q, dtype=np.float64).reshape(5, -1)
    ref = np.asarray(ref, dtype=np.float64).reshape(5, -1)
    d = q - ref
    out = {"rho": np.linalg.norm(d[0]) / np.linalg.norm(ref[0]),
           "E": np.linalg.norm(d[4]) / np.linalg.norm(ref[4])}
    mref = np.linalg.norm(ref[1:4])
    out["m"] = np.linalg.norm(d[1:4]) / mref if mref > 0 else np.linalg.norm(d[1:4])
    return out


def max_error(q, ref):
    return max(field_errors(q, ref).values())


def sigma_error(s, ref, scale):
    """L2 error of Sigma relative to max(||ref||, scale)."""
    s = np.asarray(s, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    return np.linalg.norm(s - ref) / max(np.linalg.norm(ref), scale)
