"""Seeded synthetic inputs shared by the device path, the oracle and the benchmark.

This module holds no part of the likelihood or the sampler: it builds the
frequency grid, the analytic noise PSD, Gaussian noise realisations, the
detector geometry and parameter draws.  Where an event needs an injected
signal, the caller passes its own waveform and optimal-SNR functions (the
oracle's in tests, the device library's in the benchmark), so that no signal
model lives here.  The only model fact used is that the strain amplitude
scales as 1/d_L, to place the injection at a drawn SNR.

The workloads stand in for the paper's GW150914-like analyses (Section 4),
whose strain, PSDs and waveform libraries are not available: detector count,
band, segment length, Delta f and SNR regime follow the five configurations
below.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable

import numpy as np

R_EARTH = 6.371e6  # [m], spherical Earth
N_PARAM = 11
PARAM_NAMES = ("mc", "q", "chi1", "chi2", "dl", "iota", "psi", "ra", "dec", "tc", "phic")
IDX = {n: i for i, n in enumerate(PARAM_NAMES)}

# prior kinds (unit-cube maps): 0 uniform, 1 uniform in volume, 2 sine on [0, pi], 3 cosine on [-pi/2, pi/2]
UNIFORM, VOLUME, SINE, COSINE = 0, 1, 2, 3

# Approximate Hanford-, Livingston- and Virgo-like sites, and a KAGRA-like
# fourth used only by four-detector events: latitude, longitude [deg] and
# x-arm bearing [deg from north, clockwise]; the y arm is the x arm bearing
# minus 90 deg.  Arms are perpendicular and tangent to the sphere.
SITES = {
    "H": (46.455, -119.408, 324.0),
    "L": (30.563, -90.774, 252.3),
    "V": (43.631, 10.504, 19.4),
    "K": (36.412, 137.306, 28.3),
}


def site_geometry(lat_deg: float, lon_deg: float, xbear_deg: float) -> np.ndarray:
    """[vertex xyz (m), x-arm unit vector, y-arm unit vector] in Earth-fixed axes."""
    la, lo = math.radians(lat_deg), math.radians(lon_deg)
    vertex = R_EARTH * np.array([math.cos(la) * math.cos(lo), math.cos(la) * math.sin(lo), math.sin(la)])
    east = np.array([-math.sin(lo), math.cos(lo), 0.0])
    north = np.array([-math.sin(la) * math.cos(lo), -math.sin(la) * math.sin(lo), math.cos(la)])

    def arm(b):
        b = math.radians(b)
        return math.cos(b) * north + math.sin(b) * east

    return np.concatenate([vertex, arm(xbear_deg), arm(xbear_deg - 90.0)])


def pole_geometry() -> np.ndarray:
    """A detector at the north pole with arms along the Earth-fixed x and y axes."""
    return np.array([0.0, 0.0, R_EARTH, 1.0, 0.0, 0.0, 0.0, 1.0, 0.0])


def psd_aligo(f: np.ndarray) -> np.ndarray:
    """Analytic Advanced-LIGO fit S(f) = 1e-49 [x^-4.14 - 5 x^-2 + 111 (1 - x^2 + x^4/2)/(1 + x^2/2)], x = f/215 Hz."""
    x = np.asarray(f, dtype=np.float64) / 215.0
    return 1e-49 * (x ** -4.14 - 5.0 * x ** -2 + 111.0 * (1.0 - x ** 2 + 0.5 * x ** 4) / (1.0 + 0.5 * x ** 2))


@dataclasses.dataclass
class Sampling:
    """Which of the 11 parameters are sampled, their unit-cube maps, and fixed values."""
    param_map: np.ndarray  # [D] int
    fixed: np.ndarray      # [11] values of unsampled parameters
    kind: np.ndarray       # [D] int
    lo: np.ndarray         # [D]
    hi: np.ndarray         # [D]
    periodic: np.ndarray   # [D] int

    @property
    def D(self) -> int:
        return int(len(self.param_map))


@dataclasses.dataclass
class Event:
    name: str
    freqs: np.ndarray      # [M] float64, f_low + j df
    strain: np.ndarray     # [n_det, M] complex128
    psd: np.ndarray        # [n_det, M] float64
    geom: np.ndarray       # [n_det, 9] float64
    gmst: float
    t_ref: float           # [s] from segment start (T - 2)
    fcut_mode: int         # 0 ISCO cut, 1 band only
    T: float
    theta_inj: np.ndarray  # [11]
    snr_target: float
    sampling: Sampling

    @property
    def n_det(self) -> int:
        return int(self.geom.shape[0])

    @property
    def M(self) -> int:
        return int(self.freqs.size)

    @property
    def df(self) -> float:
        return 1.0 / self.T

    def with_strain(self, strain: np.ndarray) -> "Event":
        return dataclasses.replace(self, strain=np.ascontiguousarray(strain, dtype=np.complex128))


BBH = dict(mc=(20.0, 40.0), q=(0.25, 1.0), chi=(-0.8, 0.8), dl=(400.0, 2000.0))
BNS = dict(mc=(1.1, 1.3), q=(0.7, 1.0), chi=(-0.05, 0.05), dl=(20.0, 500.0))

# The five workloads.  c1: one detector, 4 s, 20-512 Hz, zero noise, 4-D;
# c2: three detectors, 8 s, 20-1024 Hz, coloured noise, 11-D BBH (headline);
# c3: three detectors, 128 s, 20-2048 Hz, 11-D BNS (phase precision);
# c4: 64 events of {4..128} s at 20-1024 Hz, BBH or BNS; c5: c2 data, gradient.
CONFIGS = {
    "c1": dict(n_det=1, T=4.0, f_low=20.0, f_high=512.0, noise=False, source="c1", batch=1024, gmst=0.3),
    "c2": dict(n_det=3, T=8.0, f_low=20.0, f_high=1024.0, noise=True, source="bbh", batch=8192, gmst=1.7),
    "c3": dict(n_det=3, T=128.0, f_low=20.0, f_high=2048.0, noise=True, source="bns", batch=2048, gmst=1.7),
    "c5": dict(n_det=3, T=8.0, f_low=20.0, f_high=1024.0, noise=True, source="bbh", batch=4096, gmst=1.7),
}
C4_DURATIONS = (4.0, 8.0, 16.0, 32.0, 64.0, 128.0)


def grid(T: float, f_low: float, f_high: float) -> np.ndarray:
    """f_j = f_low + j/T for f_low <= f_j <= f_high (both ends included)."""
    n = int(round((f_high - f_low) * T)) + 1
    return f_low + np.arange(n, dtype=np.float64) / T


def gaussian_noise(psd: np.ndarray, T: float, rng: np.random.Generator) -> np.ndarray:
    """n_j = sqrt(S_j T / 4) (N1 + i N2), N ~ N(0, 1): <n|n> ~ chi^2 with 2M degrees of freedom."""
    s = np.sqrt(psd * T / 4.0)
    return s * (rng.standard_normal(psd.shape) + 1j * rng.standard_normal(psd.shape))


def sampling_11d(src: dict, fixed: np.ndarray) -> Sampling:
    tw = 2.0 * math.pi
    lo = np.array([src["mc"][0], src["q"][0], src["chi"][0], src["chi"][0], src["dl"][0], 0.0, 0.0, 0.0,
                   -math.pi / 2, -0.1, 0.0])
    hi = np.array([src["mc"][1], src["q"][1], src["chi"][1], src["chi"][1], src["dl"][1], math.pi, math.pi, tw,
                   math.pi / 2, 0.1, tw])
    kind = np.array([UNIFORM, UNIFORM, UNIFORM, UNIFORM, VOLUME, SINE, UNIFORM, UNIFORM, COSINE, UNIFORM, UNIFORM])
    per = np.array([0, 0, 0, 0, 0, 0, 1, 1, 0, 0, 1])
    return Sampling(np.arange(11, dtype=np.int32), np.asarray(fixed, dtype=np.float64).copy(),
                    kind.astype(np.int32), lo, hi, per.astype(np.int32))


def sampling_c1(fixed: np.ndarray) -> Sampling:
    """4-D (Mc, q, tc, phic); the other parameters stay at the injection."""
    return Sampling(np.array([IDX["mc"], IDX["q"], IDX["tc"], IDX["phic"]], dtype=np.int32),
                    np.asarray(fixed, dtype=np.float64).copy(), np.zeros(4, dtype=np.int32),
                    np.array([8.0, 0.5, -0.1, 0.0]), np.array([12.0, 1.0, 0.1, 2.0 * math.pi]),
                    np.array([0, 0, 0, 1], dtype=np.int32))


def draw_physical(src: dict, rng: np.random.Generator, n: int) -> np.ndarray:
    """n parameter vectors from the 11-D prior of a source class (isotropic sky/orientation)."""
    th = np.zeros((n, N_PARAM))
    th[:, 0] = rng.uniform(*src["mc"], n)
    th[:, 1] = rng.uniform(*src["q"], n)
    th[:, 2] = rng.uniform(*src["chi"], n)
    th[:, 3] = rng.uniform(*src["chi"], n)
    lo, hi = src["dl"]
    th[:, 4] = np.cbrt(lo ** 3 + rng.uniform(0, 1, n) * (hi ** 3 - lo ** 3))
    th[:, 5] = np.arccos(rng.uniform(-1, 1, n))
    th[:, 6] = rng.uniform(0, math.pi, n)
    th[:, 7] = rng.uniform(0, 2 * math.pi, n)
    th[:, 8] = np.arcsin(rng.uniform(-1, 1, n))
    th[:, 9] = rng.uniform(-0.1, 0.1, n)
    th[:, 10] = rng.uniform(0, 2 * math.pi, n)
    return th


WaveformFn = Callable[["Event", np.ndarray], np.ndarray]   # (event skeleton, theta[11]) -> h[n_det, M]
Snr2Fn = Callable[["Event", np.ndarray], float]            # (event skeleton, theta[11]) -> <h|h> summed over detectors


def _skeleton(name, cfg, geom, freqs, psd, theta_inj, snr_t, fcut_mode, sampling) -> Event:
    return Event(name=name, freqs=freqs, strain=np.zeros(psd.shape, dtype=np.complex128), psd=psd, geom=geom,
                 gmst=float(cfg["gmst"]), t_ref=float(cfg["T"]) - 2.0, fcut_mode=fcut_mode, T=float(cfg["T"]),
                 theta_inj=theta_inj, snr_target=snr_t, sampling=sampling)


def make_event(name: str, seed: int, waveform: WaveformFn, snr2: Snr2Fn, cfg: dict | None = None,
               fcut_mode: int = 0) -> Event:
    """Build one synthetic event: grid, PSD, noise, injection placed at a drawn SNR.

    ``waveform`` and ``snr2`` come from the caller's own side (oracle or device
    library); they receive an event skeleton with zero strain.
    """
    cfg = dict(CONFIGS[name] if cfg is None else cfg)
    rng = np.random.default_rng(seed)
    freqs = grid(cfg["T"], cfg["f_low"], cfg["f_high"])
    n_det = cfg["n_det"]
    psd = np.tile(psd_aligo(freqs), (n_det, 1))
    if cfg["source"] == "c1":
        geom = pole_geometry()[None, :]
        # F+ = 1, Fx = 0: source overhead (dec = pi/2, ra - gmst = pi/2), psi = 0, face-on; no spins.
        th = np.array([10.0, 0.8, 0.0, 0.0, 1.0, 0.0, 0.0, cfg["gmst"] + math.pi / 2, math.pi / 2, 0.0, 1.3])
        snr_t = 20.0
        sk = _skeleton(name, cfg, geom, freqs, psd, th, snr_t, fcut_mode, sampling_c1(th))
        th[4] = math.sqrt(snr2(sk, th)) / snr_t
        sampling = sampling_c1(th)
    else:
        sites = ("H", "L", "V", "K")[:n_det]
        geom = np.stack([site_geometry(*SITES[s]) for s in sites])
        src = BBH if cfg["source"] == "bbh" else BNS
        snr_t = float(rng.uniform(15.0, 30.0))
        for _ in range(10000):
            th = draw_physical(src, rng, 1)[0]
            th[9] = 0.0
            th[4] = 1.0
            sk = _skeleton(name, cfg, geom, freqs, psd, th, snr_t, fcut_mode, None)
            dl = math.sqrt(snr2(sk, th)) / snr_t
            if src["dl"][0] <= dl <= src["dl"][1]:
                th[4] = dl
                break
        else:
            raise RuntimeError("no injection with d_L inside the prior range")
        sampling = sampling_11d(src, th)
    ev = _skeleton(name, cfg, geom, freqs, psd, th, snr_t, fcut_mode, sampling)
    h = waveform(ev, th)
    n = gaussian_noise(psd, cfg["T"], rng) if cfg["noise"] else np.zeros_like(h)
    return ev.with_strain(n + h)


# Probability-probability (PP) coverage test: a fixed 4-D prior (Mc, q, tc,
# phic), injections drawn from it, the other parameters fixed; c2's network,
# segment and noise recipe.  Chosen so that the posterior is unimodal and the
# sampled prior is exactly the one the injections come from.
PP_FIXED = np.array([30.0, 0.7, 0.0, 0.0, 800.0, 0.4, 0.3, 2.7, 0.2, 0.0, 1.0])
PP_LO = np.array([25.0, 0.4, -0.05, 0.0])
PP_HI = np.array([35.0, 1.0, 0.05, 2.0 * math.pi])


def sampling_pp() -> Sampling:
    return Sampling(np.array([IDX["mc"], IDX["q"], IDX["tc"], IDX["phic"]], dtype=np.int32), PP_FIXED.copy(),
                    np.zeros(4, dtype=np.int32), PP_LO.copy(), PP_HI.copy(), np.array([0, 0, 0, 1], dtype=np.int32))


def make_pp_event(seed: int, waveform: WaveformFn) -> Event:
    """One PP injection: (Mc, q, tc, phic) drawn from the PP prior, c2's network, coloured noise."""
    cfg = dict(CONFIGS["c2"])
    rng = np.random.default_rng(10_000 + seed)
    freqs = grid(cfg["T"], cfg["f_low"], cfg["f_high"])
    psd = np.tile(psd_aligo(freqs), (3, 1))
    geom = np.stack([site_geometry(*SITES[s]) for s in ("H", "L", "V")])
    th = PP_FIXED.copy()
    th[[IDX["mc"], IDX["q"], IDX["tc"], IDX["phic"]]] = PP_LO + (PP_HI - PP_LO) * rng.uniform(0.0, 1.0, 4)
    ev = _skeleton("pp", cfg, geom, freqs, psd, th, 0.0, 0, sampling_pp())
    h = waveform(ev, th)
    return ev.with_strain(gaussian_noise(psd, cfg["T"], rng) + h)


def proposals(ev: Event, n: int, seed: int, local_fraction: float = 0.5, local_sigma: float = 1e-3) -> np.ndarray:
    """A batch of n full 11-D parameter vectors for lnL throughput runs.

    A fraction ``1 - local_fraction`` are prior draws of the sampled
    parameters; the rest perturb the injection by ``local_sigma`` times each
    sampled parameter's physical range (periodic ones wrap, others reflect).
    """
    rng = np.random.default_rng(seed + 1)
    smp = ev.sampling
    n_loc = int(round(n * local_fraction))
    n_pri = n - n_loc
    th = np.tile(smp.fixed, (n, 1))
    # prior draws of the sampled coordinates, by each coordinate's own distribution
    u = rng.uniform(0.0, 1.0, (n_pri, smp.D))
    for i, p in enumerate(smp.param_map):
        lo, hi, k = smp.lo[i], smp.hi[i], smp.kind[i]
        if k == VOLUME:
            x = np.cbrt(lo ** 3 + u[:, i] * (hi ** 3 - lo ** 3))
        elif k == SINE:
            x = np.arccos(1.0 - 2.0 * u[:, i])
        elif k == COSINE:
            x = np.arcsin(2.0 * u[:, i] - 1.0)
        else:
            x = lo + u[:, i] * (hi - lo)
        th[:n_pri, p] = x
    # local perturbations of the injection
    for i, p in enumerate(smp.param_map):
        lo, hi = smp.lo[i], smp.hi[i]
        x = ev.theta_inj[p] + local_sigma * (hi - lo) * rng.standard_normal(n_loc)
        if smp.periodic[i]:
            x = lo + np.mod(x - lo, hi - lo)
        else:
            x = np.where(x < lo, 2 * lo - x, x)
            x = np.where(x > hi, 2 * hi - x, x)
            x = np.clip(x, lo, hi)
        th[n_pri:, p] = x
    perm = rng.permutation(n)
    return np.ascontiguousarray(th[perm])


def reduced(theta_full: np.ndarray, smp: Sampling) -> np.ndarray:
    """Sampled coordinates [B, D] of full parameter vectors [B, 11]."""
    return np.ascontiguousarray(np.asarray(theta_full)[:, smp.param_map])


def c4_events(seed: int, n_events: int = 64):
    """Per-event configurations of the ragged multi-event workload (durations and source classes)."""
    rng = np.random.default_rng(seed)
    out = []
    for e in range(n_events):
        T = float(rng.choice(C4_DURATIONS))
        src = "bbh" if rng.uniform() < 0.5 else "bns"
        out.append(dict(n_det=3, T=T, f_low=20.0, f_high=1024.0, noise=True, source=src, batch=1000,
                        gmst=1.7, seed=int(rng.integers(1 << 31))))
    return out


# ---------------------------------------------------------------- calibration model
# Section 2.2: ten amplitude and ten phase nodes per interferometer.  Nodes are
# log-spaced over the analysed band; the per-node corrections are drawn from
# zero-mean Gaussians of 10 % in amplitude and 0.1 rad (about 6 degrees) in
# phase, the order of the calibration uncertainty of the LIGO detectors.
CAL_NODES = 10
CAL_SIGMA_AMP = 0.1
CAL_SIGMA_PHASE = 0.1


def cal_node_freqs(f_low: float, f_high: float, n: int = CAL_NODES) -> np.ndarray:
    """n node frequencies, log-spaced from f_low to f_high inclusive."""
    return np.geomspace(f_low, f_high, n)


def draw_calibration(rng: np.random.Generator, n: int, n_det: int, n_nodes: int = CAL_NODES,
                     sigma_amp: float = CAL_SIGMA_AMP, sigma_phase: float = CAL_SIGMA_PHASE) -> np.ndarray:
    """[n, 2 n_nodes n_det] calibration parameters: per detector dA at the nodes, then dphi [rad]."""
    out = np.empty((n, n_det, 2, n_nodes))
    out[:, :, 0, :] = sigma_amp * rng.standard_normal((n, n_det, n_nodes))
    out[:, :, 1, :] = sigma_phase * rng.standard_normal((n, n_det, n_nodes))
    return out.reshape(n, 2 * n_nodes * n_det)


def calibrated_proposals(ev: Event, n: int, seed: int, n_nodes: int = CAL_NODES) -> np.ndarray:
    """[n, 11 + 2 n_nodes n_det]: lnL throughput proposals with calibration parameters appended."""
    th = proposals(ev, n, seed)
    cal = draw_calibration(np.random.default_rng(seed + 7), n, ev.geom.shape[0], n_nodes)
    return np.ascontiguousarray(np.concatenate([th, cal], axis=1))
