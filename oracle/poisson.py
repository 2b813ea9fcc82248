"""Poisson proposal counts (paper Sec. III.D and the step J of Sec. IV.B).

The jump step draws, for each atom i, M_i ~ Poisson(mu_i) with
mu_i = n_i beta ||v_i|| L delta / 2.  The paper does not say how.  This
project's definition, used identically by the oracle and the GPU:

  * mu is split into nchunk = ceil(mu / 16) equal parts mu_c = mu / nchunk
    (FP64 division, rounded to FP32); the count is the sum of nchunk
    independent Poisson(mu_c) draws (the sum of independent Poisson variables
    is Poisson with the summed mean);
  * chunk c inverts the Poisson CDF in FP32 with its own uniform
    u = (x0 >> 8) 2^-24 from the Philox draw at slot 0x80000000 | c:
        p = exp(-mu_c); F = p; k = 0
        while u > F and k < 128:
            k += 1; p = (p * mu_c) * (1/k); F' = F + p
            if F' == F: stop;  F = F'
    (sequential search, Devroye, Non-Uniform Random Variate Generation,
    1986, Sec. X.3.2), FP32 round-to-nearest with no fused multiply-add;
  * exp(-mu_c) is this project's FP32 function expneg_f32 below, so that both
    sides compute the same bits without depending on a math library.

The FP32 CDF carries ~1e-7 relative round-off; the resulting error in the
count distribution is below 1e-6 in total variation and is stated as a
reading of the paper.

Pins: expneg_f32 against exp() in FP64 (relative error < 1e-6); counts
against scipy's Poisson quantile function away from CDF boundaries, and the
mean and variance of many draws (tests/test_oracle_rng.py).
"""
import math
import numpy as np

from . import philox

F32 = np.float32
MU_CHUNK = 16.0
K_CAP = 128

_LOG2E = F32(1.0 / math.log(2.0))
_LN2_HI = F32(0.693145751953125)
_LN2_LO = F32(math.log(2.0) - 0.693145751953125)
_TAYLOR = [F32(((-1.0) ** k) / math.factorial(k)) for k in range(8)]
_INV = np.array([F32(0.0)] + [F32(1.0) / F32(k) for k in range(1, K_CAP + 1)], dtype=np.float32)


def expneg_f32(x):
    """exp(-x) for float32 x in [0, 32], in float32 arithmetic.

    x = n ln2 + r with n = floor(x log2(e) + 1/2) and r from a two-constant
    (Cody-Waite) reduction; exp(-r) by its Taylor series to degree 7 in
    Horner form; the result is scaled by 2^-n exactly."""
    x = np.asarray(x, dtype=np.float32)
    t = x * _LOG2E
    n = np.floor(t + F32(0.5)).astype(np.float32)
    r = (x - n * _LN2_HI) - n * _LN2_LO
    p = _TAYLOR[7]
    for k in range(6, -1, -1):
        p = p * r + _TAYLOR[k]
    scale = np.ldexp(F32(1.0), -n.astype(np.int32)).astype(np.float32)
    return (p * scale).astype(np.float32)


def chunking(mu):
    """(nchunk, mu_c) for FP64 means mu >= 0 (nchunk = 0 where mu == 0)."""
    mu = np.asarray(mu, dtype=np.float64)
    nchunk = np.where(mu > 0, np.ceil(mu / MU_CHUNK), 0).astype(np.int64)
    with np.errstate(divide='ignore', invalid='ignore'):
        mu_c = np.where(nchunk > 0, mu / np.maximum(nchunk, 1), 0.0).astype(np.float32)
    return nchunk, mu_c


def invert_chunk(u, mu_c):
    """One Poisson(mu_c) count per element by FP32 sequential inversion."""
    u = np.asarray(u, dtype=np.float32)
    mu_c = np.asarray(mu_c, dtype=np.float32)
    p = expneg_f32(mu_c)
    cdf = p.copy()
    k = np.zeros(u.shape, dtype=np.int64)
    active = u > cdf
    while np.any(active):
        idx = np.nonzero(active)[0]
        k[idx] += 1
        pk = (p[idx] * mu_c[idx]) * _INV[k[idx]]
        cn = (cdf[idx] + pk).astype(np.float32)
        stalled = cn == cdf[idx]
        p[idx] = pk
        cdf[idx] = cn
        active[idx] = (~stalled) & (u[idx] > cn) & (k[idx] < K_CAP)
    return k


def counts(mu, atoms, seed, step, stream):
    """Poisson(mu_i) counts for the listed atoms (vectorised over atoms)."""
    mu = np.asarray(mu, dtype=np.float64)
    atoms = np.asarray(atoms, dtype=np.int64)
    nchunk, mu_c = chunking(mu)
    M = np.zeros(len(mu), dtype=np.int64)
    cmax = int(nchunk.max()) if len(nchunk) else 0
    for c in range(cmax):
        sel = np.nonzero(nchunk > c)[0]
        x = philox.draw(seed, philox.POISSON_SLOT | c, atoms[sel], step, stream)
        u = philox.u24(x[0]).astype(np.float32)
        M[sel] += invert_chunk(u, mu_c[sel])
    return M
