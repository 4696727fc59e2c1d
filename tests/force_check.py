"""Force comparisons shared by the GPU parity tests (FP32 GPU against the FP64
oracle on identical interaction lists).

Two bounds, both required:
- relative RMS over all 3N components, sqrt(sum |da|^2 / sum |a|^2) <= 1e-5
  (the stated tolerance of the FP32 path on identical lists);
- per particle, |da_i| <= 1e-3 (|a_i| + 1e-2 median_j |a_j|).  Every pair term
  and every local expansion carries an FP32 relative error of about 1e-6 (the
  truncation-factor fit 1.1e-6, approximate rsqrt and exp2 2^-22, FP32 offsets
  4 2^-24 sqrt(3) h / r for a pair at distance r in leaves of side h,
  accumulation sqrt(n) 2^-24); a particle's error is that times the sum of its
  terms' magnitudes, which exceeds |a_i| by the cancellation among them.  The
  floor of 1e-2 of the median force keeps particles whose force cancels to
  nearly zero (halo centres) from dividing by zero; 1e-3 leaves room for a
  cancellation factor of 100 and a close pair with h / r ~ 100.  A missing,
  doubled or mis-shifted source leaf moves the particles of the sink leaf by
  the whole contribution of that leaf, far above 1e-3 of their force.
"""
import math

import numpy as np

RMS_TOL = 1e-5
PP_TOL = 1e-3
PP_FLOOR = 1e-2


def rel_rms(a, ref):
    return math.sqrt(((a - ref) ** 2).sum() / max((ref ** 2).sum(), 1e-300))


def per_particle(a, ref, scale=None):
    """max_i |a_i - ref_i| / (|ref_i| + PP_FLOOR s), a and ref [3][n]; s = the
    median |ref| unless a force scale is given (a configuration whose forces
    cancel to zero passes the size of the terms that cancel)."""
    d = np.linalg.norm(np.asarray(a) - ref, axis=0)
    m = np.linalg.norm(ref, axis=0)
    if len(m) == 0:
        return 0.0
    s = np.median(m) if scale is None else scale
    return float((d / (m + PP_FLOOR * s + 1e-300)).max())


def assert_forces_close(a, ref, rms_tol=RMS_TOL, pp_tol=PP_TOL, scale=None):
    e, pp = rel_rms(a, ref), per_particle(a, ref, scale)
    assert e < rms_tol and pp < pp_tol, f"relative RMS {e:.3e} (bound {rms_tol}), per particle {pp:.3e} (bound {pp_tol})"
    return e, pp
