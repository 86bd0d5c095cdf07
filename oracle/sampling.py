"""Constrained-realization draws (oracle, test-only).

Sec. 2.3: with omega_1 (one standard normal per band pixel) and omega_2 (one per real
harmonic coefficient) drawn independently, the solution of A x = b,
b = P^T N^-1 d + P^T N^-1/2 omega_1 + S^-1/2 omega_2, is a sample of the posterior
p(s | d, S) = N(A^-1 P^T N^-1 d, A^-1).  A Gibbs sampler repeats such solves; the variates
are drawn here from a counter-based generator so that any sample can be reproduced from
(seed, sample) alone, on the host and on the device alike.

* Philox4x64-10 (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as
  1, 2, 3", SC'11): a 256-bit counter and a 128-bit key; each of 10 rounds replaces
  (x0, x1, x2, x3) by (hi(M1 x2) ^ x1 ^ k0, lo(M1 x2), hi(M0 x0) ^ x3 ^ k1, lo(M0 x0)),
  the key advancing by the Weyl constants between rounds.
* Variate j of stream s for (seed, sample): key (seed, sample), counter (j // 4, s, 0, 0),
  word j % 4.  A word w gives the uniform u = ((w >> 12) + 1/2) 2^-52 in (0, 1) (52 bits,
  so that u is exact in FP64); the pairs (u0, u1) and (u2, u3) of a counter give two standard normals each by the
  Box-Muller transform, z = sqrt(-2 ln u_a) (cos 2 pi u_b, sin 2 pi u_b).
* omega_2 is stream 0 over the stacked coefficient vector; omega_1 of band nu is stream
  1 + nu over that band's pixels (ring order).
* Spatially variable spectral-index mixing (Eq. Q with a power-law SED):
  q_{nu,k}(n) = m(n) (nu / nu_0)^beta(n), m the mask (0 or 1).

Parity: pinned (tests/test_oracle_sampling.py) -- the generator bit for bit against
numpy.random.Philox (the library's Philox4x64-10), the vectorised form against the
integer one, the normals against their distribution (moments, Kolmogorov-Smirnov), and the
draws' defining property: over many seeds the CR solutions of a small model have mean
A^-1 P^T N^-1 d and covariance A^-1.
"""
import numpy as np

from . import model as _model

M0 = 0xD2E7470EE14C6C93
M1 = 0xCA5A826395121157
W0 = 0x9E3779B97F4A7C15
W1 = 0xBB67AE8584CAA73B
ROUNDS = 10
_MASK64 = (1 << 64) - 1


def philox4x64_int(ctr, key, rounds=ROUNDS):
    """Philox4x64 of one counter (4 ints) and key (2 ints), Python integer arithmetic."""
    x0, x1, x2, x3 = (int(v) & _MASK64 for v in ctr)
    k0, k1 = (int(v) & _MASK64 for v in key)
    for r in range(rounds):
        if r:
            k0 = (k0 + W0) & _MASK64
            k1 = (k1 + W1) & _MASK64
        p0 = M0 * x0
        p1 = M1 * x2
        x0, x1, x2, x3 = ((p1 >> 64) ^ x1 ^ k0, p1 & _MASK64,
                          (p0 >> 64) ^ x3 ^ k1, p0 & _MASK64)
    return x0, x1, x2, x3


def _mulhilo(a, b):
    """(hi, lo) of the 128-bit products a * b of uint64 arrays, from 32-bit halves."""
    m32 = np.uint64(0xFFFFFFFF)
    s32 = np.uint64(32)
    a0, a1 = a & m32, a >> s32
    b0, b1 = b & m32, b >> s32
    p00, p01, p10, p11 = a0 * b0, a0 * b1, a1 * b0, a1 * b1
    mid = (p00 >> s32) + (p01 & m32) + (p10 & m32)
    hi = p11 + (p01 >> s32) + (p10 >> s32) + (mid >> s32)
    return hi, a * b


def philox4x64(c0, c1, c2, c3, k0, k1, rounds=ROUNDS):
    """Philox4x64 over arrays of counters (uint64 arrays of equal shape) and one key."""
    x = [np.asarray(c, dtype=np.uint64).copy() for c in (c0, c1, c2, c3)]
    k0 = np.uint64(int(k0) & _MASK64)
    k1 = np.uint64(int(k1) & _MASK64)
    m0, m1 = np.uint64(M0), np.uint64(M1)
    with np.errstate(over="ignore"):
        for r in range(rounds):
            if r:
                k0 = np.uint64((int(k0) + W0) & _MASK64)
                k1 = np.uint64((int(k1) + W1) & _MASK64)
            h0, l0 = _mulhilo(np.full_like(x[0], m0), x[0])
            h1, l1 = _mulhilo(np.full_like(x[2], m1), x[2])
            x = [h1 ^ x[1] ^ k0, l1, h0 ^ x[3] ^ k1, l0]
    return x


def words(seed, sample, stream, offset, n):
    """The uint64 words of variates offset .. offset + n - 1 of a stream."""
    if n <= 0:
        return np.zeros(0, dtype=np.uint64)
    first, last = offset // 4, (offset + n - 1) // 4
    i = np.arange(first, last + 1, dtype=np.uint64)
    z = np.zeros_like(i)
    w = philox4x64(i, np.full_like(i, np.uint64(stream)), z, z, seed, sample)
    allw = np.stack(w, axis=1).reshape(-1)          # variate 4 i + t <- word t of counter i
    start = offset - 4 * first
    return allw[start:start + n]


def uniforms(seed, sample, stream, offset, n):
    """u = ((w >> 12) + 1/2) 2^-52 for variates offset .. offset + n - 1."""
    w = words(seed, sample, stream, offset, n)
    return ((w >> np.uint64(12)).astype(np.float64) + 0.5) * 2.0 ** -52


def normals(seed, sample, stream, offset, n):
    """Standard normals (Box-Muller on the uniform pairs of each counter)."""
    if n <= 0:
        return np.zeros(0)
    first, last = offset // 4, (offset + n - 1) // 4
    u = uniforms(seed, sample, stream, 4 * first, 4 * (last - first + 1)).reshape(-1, 2)
    r = np.sqrt(-2.0 * np.log(u[:, 0]))
    z = np.stack([r * np.cos(2.0 * np.pi * u[:, 1]), r * np.sin(2.0 * np.pi * u[:, 1])],
                 axis=1).reshape(-1)
    start = offset - 4 * first
    return z[start:start + n]


def cr_omegas(model, seed, sample):
    """(omega_1 per band, omega_2) of draw `sample`."""
    w1 = [normals(seed, sample, 1 + nu, 0, model.tau[nu].size) for nu in range(model.nobs)]
    w2 = normals(seed, sample, 0, 0, model.nvec())
    return w1, w2


def cr_rhs(model, d, seed, sample):
    """b of the CR system of draw `sample` (Sec. 2.3)."""
    w1, w2 = cr_omegas(model, seed, sample)
    return _model.rhs(model, d, w1, w2)


def powerlaw_mixing(nu_ratio, beta, mask=None):
    """q(n) = m(n) (nu / nu_0)^beta(n)."""
    q = np.power(float(nu_ratio), np.asarray(beta, dtype=np.float64))
    if mask is not None:
        q = q * (np.asarray(mask) != 0)
    return q
