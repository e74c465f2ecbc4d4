"""Oracle: the random inputs of the log-coefficient field.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper draws omega_j ~ N(0, sigma^2) for the field of Sec. 5.1, Eq. (5.2)
and reuses one draw for both members of a level difference
Y_l = Q_l - Q_{l-1} (Sec. 4.1, Eq. (4.1)); it does not name a generator
(it seeds NumPy, Sec. 5.2).  The reading used throughout this project:

* xi[l][k][j] ~ N(0, 1) is the j-th KL coefficient of sample k on level l;
  sigma is folded into the basis (``oracle.kl``).
* Counter-based generator: Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
  "Parallel random numbers: as easy as 1, 2, 3", SC'11), key = (seed lo, seed
  hi), counter = (k lo, k hi, l, j >> 1).  Even j use output words (0, 1),
  odd j use words (2, 3).
* Uniform: M = (w_a << 20) | (w_b >> 12) is a 52-bit integer and
  u = (M + 1/2) * 2^-52, exact in FP64 and strictly inside (0, 1).
* Normal: z = Phi^{-1}(u) by Wichura's algorithm AS241 (PPND16, Applied
  Statistics 37 (1988) 477-484), whose tail branch needs log(); the log used
  here is written out below from the series log(m) = 2 atanh((m-1)/(m+1)).

Every floating-point operation below is a single IEEE FP64 operation (NumPy
does not contract a*b+c), in a fixed order, so that an independent
implementation doing the same operations reproduces xi bit for bit.
"""
import numpy as np

_MASK32 = np.uint64(0xFFFFFFFF)
_PHILOX_M0 = np.uint64(0xD2511F53)
_PHILOX_M1 = np.uint64(0xCD9E8D57)
_PHILOX_W0 = np.uint64(0x9E3779B9)
_PHILOX_W1 = np.uint64(0xBB67AE85)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on arrays of 32-bit words held in uint64.

    One round maps (c0, c1, c2, c3) to
    (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0));
    the key is bumped by the Weyl constants (W0, W1) between rounds.
    """
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & _MASK32 for v in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK32
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK32
    for _ in range(10):
        p0 = _PHILOX_M0 * c0          # < 2^64: exact in uint64
        p1 = _PHILOX_M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + _PHILOX_W0) & _MASK32
        k1 = (k1 + _PHILOX_W1) & _MASK32
    return c0, c1, c2, c3


def uniform_from_words(wa, wb):
    """u = (M + 1/2) 2^-52 with M = (wa << 20) | (wb >> 12), 0 <= M < 2^52."""
    wa = np.asarray(wa, dtype=np.uint64)
    wb = np.asarray(wb, dtype=np.uint64)
    m = (wa << np.uint64(20)) | (wb >> np.uint64(12))
    return (m.astype(np.float64) + 0.5) * 2.0 ** -52


# ---------------------------------------------------------------------------
# log(x) from frexp and the atanh series; ln 2 split so that e * LN2_HI is
# exact (LN2_HI holds 32 significant bits).
_LN2_HI = float.fromhex("0x1.62e42fee00000p-1")
_LN2_LO = float.fromhex("0x1.a39ef35793c76p-33")
_SQRT2 = float.fromhex("0x1.6a09e667f3bcdp+0")
# 1/(2k+1), k = 1..11, each the correctly rounded FP64 quotient.
_ATANH_C = [1.0 / (2 * k + 1) for k in range(1, 12)]


def log_series(x):
    """Natural log for 0 < x <= 1 in a fixed sequence of FP64 operations.

    x = m 2^e with m in [sqrt(1/2), sqrt(2)]; s = (m-1)/(m+1);
    log m = 2s (1 + s^2/3 + s^4/5 + ... + s^22/23)  (truncation < 2^-53);
    log x = e LN2_HI + (log m + e LN2_LO).
    """
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                      # m in [0.5, 1)
    m = m * 2.0
    e = (e - 1).astype(np.float64)
    big = m > _SQRT2
    m = np.where(big, m * 0.5, m)
    e = np.where(big, e + 1.0, e)
    f = m - 1.0
    s = f / (m + 1.0)
    z = s * s
    p = np.full_like(z, _ATANH_C[-1])
    for c in reversed(_ATANH_C[:-1]):
        p = p * z
        p = p + c
    t = s + s
    zp = z * p
    lm = t * zp
    lm = t + lm
    lo = e * _LN2_LO
    lm = lm + lo
    hi = e * _LN2_HI
    return hi + lm


# ---------------------------------------------------------------------------
# AS241 (PPND16): rational approximations of Phi^{-1}, relative accuracy ~1e-16.
_A = [3.3871328727963666080e0, 1.3314166789178437745e+2, 1.9715909503065514427e+3,
      1.3731693765509461125e+4, 4.5921953931549871457e+4, 6.7265770927008700853e+4,
      3.3430575583588128105e+4, 2.5090809287301226727e+3]
_B = [1.0, 4.2313330701600911252e+1, 6.8718700749205790830e+2, 5.3941960214247511077e+3,
      2.1213794301586595867e+4, 3.9307895800092710610e+4, 2.8729085735721942674e+4,
      5.2264952788528545610e+3]
_C = [1.42343711074968357734e0, 4.63033784615654529590e0, 5.76949722146069140550e0,
      3.64784832476320460504e0, 1.27045825245236838258e0, 2.41780725177450611770e-1,
      2.27238449892691845833e-2, 7.74545014278341407640e-4]
_D = [1.0, 2.05319162663775882187e0, 1.67638483018380384940e0, 6.89767334985100004550e-1,
      1.48103976427480074590e-1, 1.51986665636164571966e-2, 5.47593808499534494600e-4,
      1.05075007164441684324e-9]
_E = [6.65790464350110377720e0, 5.46378491116411436990e0, 1.78482653991729133580e0,
      2.96560571828504891230e-1, 2.65321895265761230930e-2, 1.24266094738807843860e-3,
      2.71155556874348757815e-5, 2.01033439929228813265e-7]
_F = [1.0, 5.99832206555887937690e-1, 1.36929880922735805310e-1, 1.48753612908506148525e-2,
      7.86869131145613259100e-4, 1.84631831751005468180e-5, 1.42151175831644588870e-7,
      2.04426310338993978564e-15]
_SPLIT1 = 0.425
_SPLIT2 = 5.0
_CONST1 = 0.180625
_CONST2 = 1.6


def _horner(coef, r):
    """coef[7] r^7 + ... + coef[0], evaluated as p = p*r; p = p + c."""
    p = np.full_like(r, coef[7])
    for c in reversed(coef[:7]):
        p = p * r
        p = p + c
    return p


def normal_from_uniform(u):
    """z = Phi^{-1}(u) by AS241; u strictly inside (0, 1)."""
    u = np.asarray(u, dtype=np.float64)
    q = u - 0.5
    z = np.empty_like(u)
    central = np.abs(q) <= _SPLIT1
    if central.any():
        qc = q[central]
        r = _CONST1 - qc * qc
        num = qc * _horner(_A, r)
        z[central] = num / _horner(_B, r)
    tail = ~central
    if tail.any():
        qt = q[tail]
        ut = u[tail]
        r = np.where(qt < 0.0, ut, 1.0 - ut)
        r = np.sqrt(-log_series(r))
        zt = np.empty_like(r)
        near = r <= _SPLIT2
        if near.any():
            rn = r[near] - _CONST2
            zt[near] = _horner(_C, rn) / _horner(_D, rn)
        far = ~near
        if far.any():
            rf = r[far] - _SPLIT2
            zt[far] = _horner(_E, rf) / _horner(_F, rf)
        z[tail] = np.where(qt < 0.0, -zt, zt)
    return z


def draw_xi(seed, level, first, count, K):
    """xi[k - first][j] for samples k in [first, first + count) of level l, j < K."""
    k = np.uint64(first) + np.arange(count, dtype=np.uint64)
    j = np.arange(K, dtype=np.uint64)
    kk, jj = np.meshgrid(k, j, indexing="ij")
    seed = int(seed)
    w0, w1, w2, w3 = philox4x32_10(kk & _MASK32, kk >> np.uint64(32),
                                   np.full_like(kk, np.uint64(level)), jj >> np.uint64(1),
                                   np.uint64(seed & 0xFFFFFFFF), np.uint64((seed >> 32) & 0xFFFFFFFF))
    odd = (jj & np.uint64(1)).astype(bool)
    wa = np.where(odd, w2, w0)
    wb = np.where(odd, w3, w1)
    return normal_from_uniform(uniform_from_words(wa, wb)).reshape(count, K)
