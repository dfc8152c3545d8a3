"""Seeded synthetic event samples shaped like the paper's pseudo-experiments.

This module is the ONE piece shared by the oracle side and the CUDA side: it only
draws events.  It holds none of the likelihood arithmetic (no normalisation, no log,
no gradient); the densities below are used only as accept-reject targets.

Random numbers come from a counter-based SplitMix64 (Steele, Lea & Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014): value k of a stream is
mix(state0 + k * gamma), so any slice of a stream can be drawn independently and the
same seed gives the same events on every machine.  The base seed 229387429 is the one
the paper's example control file uses (paper appendix, mass-fit control file).

Workloads (paper Sec. 3; units MeV for the default configurations):
  * mass model (Sec. 3.2, Eq. 2): Gaussian signal + exponential background on a window;
  * 4D B0 -> K*0 mu mu model: Gaussian x angular rate (Sec. 2.4.2, Eq. 3) for signal,
    exponential x second-order Chebyshev in each angle for background;
  * toy ensembles with Poisson-distributed event counts, in CSR layout.
Generation is accept-reject as in the paper (Sec. 2.5), component by component.
"""
import math

import numpy as np

BASE_SEED = 229387429

MASS1D = 1
KSTAR4D = 2

# default (MeV) configuration
MASS_WINDOW = (5170.0, 5970.0)
RANGES_1D = np.array(MASS_WINDOW)
RANGES_4D = np.array([MASS_WINDOW[0], MASS_WINDOW[1], -1.0, 1.0, -1.0, 1.0, -math.pi, math.pi])

PARAMS_1D = ["mu", "sigma", "alpha", "fsig"]
PARAMS_4D = ["mu", "sigma", "FL", "S3", "S4", "S5", "AFB", "S7", "S8", "S9",
             "alpha", "c1_ctl", "c2_ctl", "c1_ctk", "c2_ctk", "c1_phi", "c2_phi", "fsig"]

TRUTH_1D = np.array([5279.6, 20.0, -0.002, 0.3])
TRUTH_4D = np.array([5279.6, 20.0, 0.7, -0.01, -0.08, -0.05, -0.1, 0.02, 0.01, -0.01,
                     -0.002, -0.10, 0.05, 0.20, -0.10, 0.00, 0.05, 0.5])

# the paper's own mass-fit set (GeV units, Table of generation values in Sec. 3.2)
RANGES_1D_GEV = np.array([5.0, 7.0])
TRUTH_1D_GEV = np.array([5.28, 0.06, -1.0, 0.3])

_M64 = (1 << 64) - 1
_BATCH = 1 << 23  # largest candidate batch of the accept-reject loops
_GAMMA = 0x9E3779B97F4A7C15


def _mix_int(z: int) -> int:
    z &= _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


class Stream:
    """Counter-based SplitMix64 stream: value k = mix(state0 + (k+1) * gamma)."""

    def __init__(self, seed: int = BASE_SEED, stream: int = 0):
        self.state0 = _mix_int((seed & _M64) ^ _mix_int((stream * _GAMMA + 1) & _M64))
        self.counter = 0

    def u64(self, n: int) -> np.ndarray:
        k = np.arange(self.counter + 1, self.counter + n + 1, dtype=np.uint64)
        self.counter += n
        with np.errstate(over="ignore"):
            return _mix(np.uint64(self.state0) + k * np.uint64(_GAMMA))

    def uniform(self, n: int) -> np.ndarray:
        """Doubles in the open interval (0, 1): ((x >> 11) + 1/2) * 2^-53."""
        return ((self.u64(n) >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


# ---------------------------------------------------------------------------------
# component samplers
# ---------------------------------------------------------------------------------
def _gauss_trunc(rs: Stream, n: int, mu: float, sigma: float, lo: float, hi: float) -> np.ndarray:
    out = np.empty(0)
    while len(out) < n:
        k = min(max(2 * (n - len(out)), 64), _BATCH)
        u1, u2 = rs.uniform(k), rs.uniform(k)
        z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)  # Box-Muller
        m = mu + sigma * z
        out = np.concatenate([out, m[(m >= lo) & (m <= hi)]])
    return out[:n]


def _expo_trunc(rs: Stream, n: int, alpha: float, lo: float, hi: float) -> np.ndarray:
    u = rs.uniform(n)
    if alpha == 0.0:
        return lo + u * (hi - lo)
    return lo + np.log1p(u * np.expm1(alpha * (hi - lo))) / alpha  # inverse CDF


def _cheb_trunc(rs: Stream, n: int, c1: float, c2: float) -> np.ndarray:
    """x in [-1, 1] with density proportional to 1 + c1 x + c2 (2x^2 - 1)."""
    bound = 1.0 + abs(c1) + abs(c2)
    out = np.empty(0)
    while len(out) < n:
        k = min(max(2 * (n - len(out)), 64), _BATCH)
        x = 2.0 * rs.uniform(k) - 1.0
        y = bound * rs.uniform(k)
        dens = 1.0 + c1 * x + c2 * (2.0 * x * x - 1.0)
        out = np.concatenate([out, x[y < dens]])
    return out[:n]


def _angular_density(ctl, ctk, phi, ang):
    """Angular decay rate used as the accept-reject target (paper Eq. 3)."""
    FL, S3, S4, S5, AFB, S7, S8, S9 = ang
    sl2, sk2 = 1.0 - ctl ** 2, 1.0 - ctk ** 2
    sl, sk = np.sqrt(sl2), np.sqrt(sk2)
    c2l = 2.0 * ctl ** 2 - 1.0
    s2l, s2k = 2.0 * sl * ctl, 2.0 * sk * ctk
    r = ((1 - FL) * 0.75 * sk2 + FL * ctk ** 2 + (1 - FL) * 0.25 * sk2 * c2l - FL * ctk ** 2 * c2l
         + S3 * sk2 * sl2 * np.cos(2 * phi) + S4 * s2k * s2l * np.cos(phi) + S5 * s2k * sl * np.cos(phi)
         + AFB * (4.0 / 3.0) * sk2 * ctl + S7 * s2k * sl * np.sin(phi) + S8 * s2k * s2l * np.sin(phi)
         + S9 * sk2 * sl2 * np.sin(2 * phi))
    return 9.0 / (32.0 * math.pi) * r


def _angles_signal(rs: Stream, n: int, ang) -> tuple:
    FL, S3, S4, S5, AFB, S7, S8, S9 = ang
    # accept-reject bound of the paper's angular PDF (appendix, get_max of the user PDF)
    bound = 9.0 / (32.0 * math.pi) * (4.0 + abs(S3) + abs(S4) + abs(S5) + 4.0 / 3.0 * abs(AFB)
                                     + abs(S7) + abs(S8) + abs(S9))
    acc = [np.empty(0)] * 3
    have = 0
    while have < n:
        k = min(max(12 * (n - have), 256), _BATCH)
        ctl = 2.0 * rs.uniform(k) - 1.0
        ctk = 2.0 * rs.uniform(k) - 1.0
        phi = math.pi * (2.0 * rs.uniform(k) - 1.0)
        y = bound * rs.uniform(k)
        keep = y < _angular_density(ctl, ctk, phi, ang)
        acc = [np.concatenate([a, b[keep]]) for a, b in zip(acc, (ctl, ctk, phi))]
        have = len(acc[0])
    return tuple(a[:n] for a in acc)


# ---------------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------------
def mass1d(n: int, seed: int = BASE_SEED, stream: int = 0, theta=TRUTH_1D, ranges=RANGES_1D):
    """n events of the mass model; returns [m] (list of one column)."""
    mu, sigma, alpha, fsig = (float(t) for t in theta)
    lo, hi = float(ranges[0]), float(ranges[1])
    rs = Stream(seed, stream)
    is_sig = rs.uniform(n) < fsig
    ns = int(is_sig.sum())
    m = np.empty(n)
    m[is_sig] = _gauss_trunc(rs, ns, mu, sigma, lo, hi)
    m[~is_sig] = _expo_trunc(rs, n - ns, alpha, lo, hi)
    return [m]


def kstar4d(n: int, seed: int = BASE_SEED, stream: int = 0, theta=TRUTH_4D, ranges=RANGES_4D):
    """n events of the 4D model; returns [m, ctl, ctk, phi]."""
    th = [float(t) for t in theta]
    mu, sigma = th[0], th[1]
    ang = th[2:10]
    alpha = th[10]
    cheb = th[11:17]
    fsig = th[17]
    lo, hi = float(ranges[0]), float(ranges[1])
    rs = Stream(seed, stream)
    is_sig = rs.uniform(n) < fsig
    ns = int(is_sig.sum())
    nb = n - ns
    m = np.empty(n)
    ctl = np.empty(n)
    ctk = np.empty(n)
    phi = np.empty(n)
    m[is_sig] = _gauss_trunc(rs, ns, mu, sigma, lo, hi)
    a, b, c = _angles_signal(rs, ns, ang)
    ctl[is_sig], ctk[is_sig], phi[is_sig] = a, b, c
    m[~is_sig] = _expo_trunc(rs, nb, alpha, lo, hi)
    ctl[~is_sig] = _cheb_trunc(rs, nb, cheb[0], cheb[1])
    ctk[~is_sig] = _cheb_trunc(rs, nb, cheb[2], cheb[3])
    phi[~is_sig] = math.pi * _cheb_trunc(rs, nb, cheb[4], cheb[5])
    return [m, ctl, ctk, phi]


def weights(n: int, seed: int = BASE_SEED, stream: int = 1000003, lo: float = 0.5, hi: float = 1.5):
    """Per-event weights w ~ Uniform(lo, hi)."""
    return lo + (hi - lo) * Stream(seed, stream).uniform(n)


def poisson(n: int, lam: float, seed: int = BASE_SEED, stream: int = 7) -> np.ndarray:
    """n Poisson(lam) counts by inversion of the cumulative distribution."""
    kmax = int(lam + 20.0 * math.sqrt(lam) + 20)
    k = np.arange(kmax + 1, dtype=np.float64)
    logp = k * math.log(lam) - lam - np.array([math.lgamma(x + 1.0) for x in k])
    cdf = np.cumsum(np.exp(logp))
    u = Stream(seed, stream).uniform(n)
    return np.minimum(np.searchsorted(cdf, u * cdf[-1]), kmax).astype(np.int64)


def toys4d(n_toys: int, mean_events: float = 2000.0, seed: int = BASE_SEED, theta=TRUTH_4D,
           ranges=RANGES_4D):
    """Toy ensemble in CSR layout: (offsets[n_toys+1], [m, ctl, ctk, phi]) with Poisson sizes."""
    counts = poisson(n_toys, mean_events, seed, stream=7)
    offsets = np.zeros(n_toys + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(counts)
    cols = [np.empty(int(offsets[-1])) for _ in range(4)]
    for t in range(n_toys):
        ev = kstar4d(int(counts[t]), seed, stream=100000 + t, theta=theta, ranges=ranges)
        for c in range(4):
            cols[c][offsets[t]:offsets[t + 1]] = ev[c]
    return offsets, cols


def toys1d(n_toys: int, mean_events: float = 1000.0, seed: int = BASE_SEED, theta=TRUTH_1D,
           ranges=RANGES_1D, fixed_size: bool = False):
    """Toy ensemble of the mass model in CSR layout: (offsets, [m])."""
    if fixed_size:
        counts = np.full(n_toys, int(mean_events), dtype=np.int64)
    else:
        counts = poisson(n_toys, mean_events, seed, stream=8)
    offsets = np.zeros(n_toys + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(counts)
    m = np.empty(int(offsets[-1]))
    for t in range(n_toys):
        m[offsets[t]:offsets[t + 1]] = mass1d(int(counts[t]), seed, stream=200000 + t, theta=theta,
                                               ranges=ranges)[0]
    return offsets, [m]


def perturb(theta, scale, seed: int = BASE_SEED, k: int = 0, frac: float = 0.5) -> np.ndarray:
    """theta + frac * scale * z with z uniform in [-sqrt3, sqrt3] (unit variance), draw k."""
    th = np.asarray(theta, dtype=float)
    z = (2.0 * Stream(seed, 300000 + k).uniform(len(th)) - 1.0) * math.sqrt(3.0)
    return th + frac * np.asarray(scale, dtype=float) * z
