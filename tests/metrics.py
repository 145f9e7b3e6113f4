"""Error metrics shared by the parity tests: relative L2 per conserved field
(rho, m_x, m_y, m_z, E), each against its own reference norm."""
import numpy as np

FIELDS = ("rho", "mx", "my", "mz", "E")

# A momentum component whose reference norm is below this fraction of the
# momentum vector's norm carries no scale of its own (a component that is
# zero by symmetry, e.g. m_y of a flow along x): its error is measured
# against the vector's norm instead.
COMPONENT_FLOOR = 1e-3


def field_errors(q, ref):
    """Relative L2 error of each conserved field of a (5, ...) state against
    a reference: ||q_v - ref_v||_2 / ||ref_v||_2 for v in FIELDS. A momentum
    component with ||ref_v|| < COMPONENT_FLOOR ||ref_m|| is divided by
    ||ref_m|| instead; with ||ref_m|| = 0 the error is absolute."""
    q = np.asarray(q, dtype=np.float64).reshape(5, -1)
    ref = np.asarray(ref, dtype=np.float64).reshape(5, -1)
    d = q - ref
    mref = np.linalg.norm(ref[1:4])
    out = {}
    for v, name in enumerate(FIELDS):
        den = np.linalg.norm(ref[v])
        if 1 <= v <= 3 and den < COMPONENT_FLOOR * mref:
            den = mref
        out[name] = np.linalg.norm(d[v]) / den if den > 0 else np.linalg.norm(d[v])
    return out


def field_errors_torch(q, ref):
    """field_errors for (5, ...) torch tensors on any device, evaluated there
    in FP64 (for states too large to copy to the host)."""
    import torch
    q = q.reshape(5, -1)
    ref = ref.reshape(5, -1)
    mref = float(torch.linalg.vector_norm(ref[1:4].double()))
    out = {}
    for v, name in enumerate(FIELDS):
        num = float(torch.linalg.vector_norm(q[v].double() - ref[v].double()))
        den = float(torch.linalg.vector_norm(ref[v].double()))
        if 1 <= v <= 3 and den < COMPONENT_FLOOR * mref:
            den = mref
        out[name] = num / den if den > 0 else num
    return out


def max_error(q, ref):
    return max(field_errors(q, ref).values())


def sigma_error(s, ref, scale):
    """L2 error of Sigma relative to max(||ref||, scale)."""
    s = np.asarray(s, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    return np.linalg.norm(s - ref) / max(np.linalg.norm(ref), scale)
