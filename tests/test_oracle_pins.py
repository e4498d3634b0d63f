"""Pins of the FP64 oracle against facts fixed outside it (CPU only).

Each check ties the oracle to something other than itself: closed forms of the
noise-weighted inner product, textbook post-Newtonian and antenna-pattern
formulas written in an independent form, library routines (FFT, erf, mpmath),
invariances, finite differences, the paper's Eq. 5 and Table 1, and the
closed-form evidence of a Gaussian likelihood in a box.  The tests are chosen
so that a dropped factor, a wrong sign or a transposed index in the oracle
fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import special, stats

import oracle
from paper_1909_11873_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
TSUN = 4.925490947e-6


def wf(ev, th):
    return oracle.waveform(ev, th)


def snr2(ev, th):
    return -2.0 * oracle.loglike(ev.with_strain(np.zeros_like(ev.strain)), th[None])[0]


@pytest.fixture(scope="module")
def c1():
    return I.make_event("c1", 11, wf, snr2)


@pytest.fixture(scope="module")
def c2():
    return I.make_event("c2", 12, wf, snr2)


def inner(ev, a, b):
    """<a|b> summed over detectors, from the definition 4 df Re sum conj(a) b / S."""
    return float(np.sum(4.0 * ev.df * np.real(np.conj(a) * b) / ev.psd))


# ---------------------------------------------------------------- noise / inner product
def test_noise_inner_product_is_chi2_2M(c1):
    """<n|n> ~ chi^2 with 2M degrees of freedom (mean 2M, variance 4M)."""
    rng = np.random.default_rng(0)
    vals = [inner(c1, n, n) for n in (I.gaussian_noise(c1.psd, c1.T, rng) for _ in range(400))]
    M = c1.M
    assert abs(np.mean(vals) - 2 * M) < 4 * math.sqrt(4 * M / 400)
    assert abs(np.var(vals) / (4 * M) - 1) < 0.25


def test_lnl_at_truth_with_noise_is_gaussian(c1):
    """lnL(theta_true; n + h) = <n|h> + rho^2/2 with <n|h> ~ N(0, rho^2) over noise draws."""
    h = oracle.waveform(c1, c1.theta_inj)
    rho2 = inner(c1, h, h)
    rng = np.random.default_rng(1)
    vals = []
    for _ in range(300):
        ev = c1.with_strain(h + I.gaussian_noise(c1.psd, c1.T, rng))
        vals.append(oracle.loglike(ev, c1.theta_inj[None])[0])
    vals = np.array(vals)
    assert abs(vals.mean() - rho2 / 2) < 4 * math.sqrt(rho2 / 300)
    assert abs(vals.var() / rho2 - 1) < 0.3


def test_zero_noise_lnl_is_half_snr2(c1):
    """Zero-noise injection: lnL(truth) = rho^2/2, lnL against empty data = -rho^2/2, rho = 20."""
    l_truth = oracle.loglike(c1, c1.theta_inj[None])[0]
    l_empty = oracle.loglike(c1.with_strain(np.zeros_like(c1.strain)), c1.theta_inj[None])[0]
    assert l_truth == pytest.approx(200.0, rel=1e-12)
    assert l_empty == pytest.approx(-200.0, rel=1e-12)


def test_newtonian_snr_textbook_si_units(c1):
    """Optimal SNR from the textbook Newtonian amplitude in SI units (G, c, M_sun, pc),
    |h| = sqrt(5/24) pi^(-2/3) (G Mc)^(5/6) / (c^(3/2) dL) f^(-7/6), overhead optimal source.
    Checks the amplitude constant, the exponents and 4 df / S."""
    G, c, msun, pc = 6.67430e-11, 299792458.0, 1.98840987e30, 3.085677581491367e16
    th = c1.theta_inj.copy()
    mc = th[0] * msun
    dl = th[4] * 1e6 * pc
    eta = th[1] / (1 + th[1]) ** 2
    mtot_s = th[0] * eta ** -0.6 * G * msun / c ** 3
    f_isco = 1.0 / (6 ** 1.5 * math.pi * mtot_s)
    f = c1.freqs[c1.freqs <= f_isco]
    S = c1.psd[0, : f.size]
    amp = math.sqrt(5 / 24) * math.pi ** (-2 / 3) * (G * mc) ** (5 / 6) / (c ** 1.5 * dl) * f ** (-7 / 6)
    rho2 = np.sum(4 * c1.df * amp ** 2 / S)
    # G Msun/c^3 in SI differs from the oracle's T_sun constant by ~1e-9 relative
    assert -2 * oracle.loglike(c1.with_strain(np.zeros_like(c1.strain)), th[None])[0] == pytest.approx(rho2, rel=1e-6)


def test_hh_independent_of_phase_parameters(c2):
    """<h|h> depends on amplitude parameters only: spins, tc and phic move the phase alone."""
    ev0 = c2.with_strain(np.zeros_like(c2.strain))
    base = c2.theta_inj.copy()
    ths = np.tile(base, (4, 1))
    ths[1, 2:4] = [0.5, -0.3]
    ths[2, 9] = 0.05
    ths[3, 10] = 2.0
    # keep the ISCO cut (set by the masses alone) unchanged
    l = oracle.loglike(ev0, ths)
    assert np.allclose(l, l[0], rtol=1e-12, atol=0)


# ---------------------------------------------------------------- phase / time structure
def test_phic_sweep_is_a_pure_sinusoid(c2):
    """lnL(phic) = |z| cos(phic - arg z) - <h|h>/2: fit A cos + B sin + C, residual at rounding."""
    phis = np.linspace(0, 2 * math.pi, 25, endpoint=False)
    ths = np.tile(c2.theta_inj, (phis.size, 1))
    ths[:, 0] *= 1.0003  # slightly off the injection so <d|h> is not at its peak
    ths[:, 10] = phis
    l = oracle.loglike(c2, ths)
    X = np.stack([np.cos(phis), np.sin(phis), np.ones_like(phis)], axis=1)
    coef, *_ = np.linalg.lstsq(X, l, rcond=None)
    assert np.max(np.abs(X @ coef - l)) < 1e-9 * np.max(np.abs(l))
    hh = -2 * oracle.loglike(c2.with_strain(np.zeros_like(c2.strain)), ths[:1])[0]
    assert coef[2] == pytest.approx(-hh / 2, rel=1e-10)


def test_tc_sweep_matches_fft(c1):
    """z(tc) = sum_j w_j conj(d_j) h_j(tc=0) e^{-2 pi i f_j tc}: lnL on the grid tc_k = k/(N df)
    equals Re[e^{-2 pi i f_0 tc_k} FFT(x)_k] - <h|h>/2 (numpy FFT as the library routine)."""
    th0 = c1.theta_inj.copy()
    th0[0] = 10.02  # template off the injection
    th0[9] = 0.0
    h0 = oracle.waveform(c1, th0)[0]
    d = c1.strain[0]
    x = 4 * c1.df * np.conj(d) * h0 / c1.psd[0]
    N = 8192
    X = np.fft.fft(x, n=N)
    ks = np.array([1, 3, 17, 40, 200, N - 50, N - 7])
    tck = ks / (N * c1.df)
    tck = np.where(tck > 0.5 * N / (N * c1.df), tck - 1.0 / c1.df, tck)  # map to (-T/2, T/2]
    ths = np.tile(th0, (ks.size, 1))
    ths[:, 9] = tck
    hh = np.sum(4 * c1.df * np.abs(h0) ** 2 / c1.psd[0])
    pred = np.real(np.exp(-2j * math.pi * c1.freqs[0] * tck) * X[ks]) - hh / 2
    got = oracle.loglike(c1, ths)
    assert np.allclose(got, pred, rtol=0, atol=1e-9 * hh)


def test_time_and_phase_shift_invariance(c1):
    """Shifting injection and template tc (or phic) together leaves zero-noise lnL unchanged."""
    th_t = c1.theta_inj.copy()
    th_t[0] = 10.01
    th_t[1] = 0.79
    base = oracle.loglike(c1, th_t[None])[0]
    for key, delta in ((9, 0.037), (10, 0.9)):
        inj = c1.theta_inj.copy()
        inj[key] += delta
        ev = c1.with_strain(oracle.waveform(c1, inj))
        tt = th_t.copy()
        tt[key] += delta
        assert oracle.loglike(ev, tt[None])[0] == pytest.approx(base, abs=1e-9)


def test_newtonian_and_1pn_phase_coefficients_textbook():
    """Psi_PN * 128 eta v^5 / 3 = 1 + phi2 v^2 + phi3 v^3 + ... : extract phi2, phi3 at small v and
    compare with the textbook non-spinning values 3715/756 + 55 eta/9 and -16 pi."""
    mc, q = 1.2, 0.8
    eta = q / (1 + q) ** 2
    M = mc * eta ** -0.6 * TSUN
    for v in (1e-4,):
        f = v ** 3 / (math.pi * M)
        g = oracle.pn_psi(mc, q, 0.0, 0.0, f) * 128 * eta * v ** 5 / 3 - 1.0
        phi2 = 3715 / 756 + 55 * eta / 9
        assert g / v ** 2 == pytest.approx(phi2, rel=1e-3)
        phi3 = (g - phi2 * v ** 2) / v ** 3
        assert phi3 == pytest.approx(-16 * math.pi, rel=2e-3)


@pytest.mark.parametrize("q", [1.0, 0.8, 0.35])
def test_nonspinning_phase_series_to_3_5pn_published_coefficients(q):
    """The oracle's non-spinning TaylorF2 phase through 3.5PN against the published coefficients
    (Arun, Iyer, Sathyaprakash & Sundararajan 2005; Buonanno, Iyer, Ochsner, Pan & Sathyaprakash
    2009): Psi * 128 eta v^5 / 3 - 1 is exactly a combination of v^2 .. v^7, v^5 ln v and v^6 ln v,
    so a least-squares fit over v in [0.05, 0.4] recovers each coefficient -- phi2, phi3 = -16 pi,
    phi4, the 2.5PN term phi5 (1 + 3 ln(v / v_lso)) with v_lso = 6^{-1/2}, the 3PN term with
    -6848/21 ln(4 v), and phi7 -- and every eta polynomial is checked at three mass ratios."""
    mc = 1.2
    eta = q / (1 + q) ** 2
    M = mc * eta ** -0.6 * TSUN
    v = np.linspace(0.05, 0.4, 40)
    f = v ** 3 / (math.pi * M)
    g = np.array([oracle.pn_psi(mc, q, 0.0, 0.0, fi) for fi in f]) * 128 * eta * v ** 5 / 3 - 1.0
    A = np.stack([v ** 2, v ** 3, v ** 4, v ** 5, v ** 5 * np.log(v), v ** 6, v ** 6 * np.log(v), v ** 7], axis=1)
    scale = np.abs(A).max(axis=0)
    coef = np.linalg.lstsq(A / scale, g, rcond=None)[0] / scale
    euler_gamma = 0.5772156649015329
    phi5 = math.pi * (38645 / 756 - 65 * eta / 9)
    published = [
        3715 / 756 + 55 * eta / 9,
        -16 * math.pi,
        15293365 / 508032 + 27145 * eta / 504 + 3085 * eta ** 2 / 72,
        phi5 * (1 + 1.5 * math.log(6)),
        3 * phi5,
        11583231236531 / 4694215680 - 640 * math.pi ** 2 / 3 - 6848 * euler_gamma / 21
        - 6848 / 21 * math.log(4) + (-15737765635 / 3048192 + 2255 * math.pi ** 2 / 12) * eta
        + 76055 * eta ** 2 / 1728 - 127825 * eta ** 3 / 1296,
        -6848 / 21,
        math.pi * (77096675 / 254016 + 378515 * eta / 1512 - 74045 * eta ** 2 / 756),
    ]
    assert coef == pytest.approx(published, rel=1e-8)


def test_spin_orbit_and_spin_spin_terms_textbook_form():
    """1.5PN spin-orbit written as (113/3 - 76 eta/3) chi_s + (113/3) delta chi_a and 2PN aligned
    spin-spin as -10 eta (721/48 - 247/48) chi1 chi2: extracted from the oracle's series."""
    mc, q, c1, c2 = 1.2, 0.6, 0.4, -0.3
    eta = q / (1 + q) ** 2
    delta = math.sqrt(1 - 4 * eta)
    chis, chia = (c1 + c2) / 2, (c1 - c2) / 2
    M = mc * eta ** -0.6 * TSUN
    v = 1e-4
    f = v ** 3 / (math.pi * M)
    k = 128 * eta * v ** 5 / 3
    g_spin = oracle.pn_psi(mc, q, c1, c2, f) * k
    g_none = oracle.pn_psi(mc, q, 0.0, 0.0, f) * k
    so = (113 / 3 - 76 * eta / 3) * chis + 113 / 3 * delta * chia
    assert (g_spin - g_none) / v ** 3 == pytest.approx(so, rel=2e-3)
    # spin-spin at 2PN: every other spin term is linear in the spins, so the symmetric
    # combination g(chi) + g(-chi) - 2 g(0) keeps only the chi1 chi2 term
    v = 1e-2
    f = v ** 3 / (math.pi * M)
    k = 128 * eta * v ** 5 / 3
    d4 = 0.5 * (oracle.pn_psi(mc, q, c1, c2, f) + oracle.pn_psi(mc, q, -c1, -c2, f)
                - 2 * oracle.pn_psi(mc, q, 0.0, 0.0, f)) * k
    ss = -10 * eta * (721 / 48 - 247 / 48) * c1 * c2
    assert d4 / v ** 4 == pytest.approx(ss, rel=1e-5)


def _taylorf2_from_energy_and_flux(q, chi1, chi2):
    """phi_k of Psi * 128 eta v^5 / 3 = sum phi_k v^k (k != 5) and the v^5 ln v coefficient L5,
    derived from the binding energy and the energy flux by the stationary-phase approximation.

    E(v) = -(eta v^2 / 2) e(v) and F(v) = (32/5) eta^2 v^10 f(v) with v = (pi M f)^(1/3), M = 1.  The
    orbit obeys dt/dv = -E'(v) / F(v) and d(phi_orb)/dt = v^3; the stationary point of the dominant
    harmonic gives Psi(f) = 2 pi f t(v_f) - 2 phi_orb(v_f) - pi/4, i.e. up to terms linear in f and
    constants Psi = 2 int_{v_f} (v_f^3 - v^3) E'(v)/F(v) dv.  Writing E'/F = -(5 / (32 eta)) v^-9 *
    sum a_k v^k, the lower limit of the v^k term gives (15 / (16 eta)) a_k v_f^(k-5) / ((k-8)(k-5)),
    so phi_k = 40 a_k / ((k-8)(k-5)); at k = 5 it gives -(5 / (16 eta)) a_5 ln v_f, so L5 = -(40/3) a_5.

    Energy and flux: the non-spinning terms through 2PN and the 1.5PN tail of the flux, and the
    spin-orbit terms -- energy at 1.5, 2.5 and 3.5PN, flux at 1.5, 2.5, 3 (tail) and 3.5PN --
    in the spin variables S = m1^2 chi1 + m2^2 chi2 and Sigma = M (m2 chi2 - m1 chi1) (masses in
    units of M), as collected in Blanchet's review (Living Rev. Relativ. 17, 2, 2014), from
    Blanchet, Buonanno & Faye (2006, 2011) and Bohe, Marsat, Faye & Blanchet (2013)."""
    x1, x2 = 1.0 / (1.0 + q), q / (1.0 + q)
    eta, d = x1 * x2, x1 - x2
    S, Sg = x1 * x1 * chi1 + x2 * x2 * chi2, x2 * chi2 - x1 * chi1
    pi = math.pi
    e = np.zeros(8)
    e[0] = 1.0
    e[2] = -0.75 - eta / 12
    e[3] = 14 / 3 * S + 2 * d * Sg
    e[4] = -27 / 8 + 19 / 8 * eta - eta ** 2 / 24
    e[5] = (11 - 61 / 9 * eta) * S + d * (3 - 10 / 3 * eta) * Sg
    e[7] = (135 / 4 - 367 / 4 * eta + 29 / 12 * eta ** 2) * S + d * (27 / 4 - 39 * eta + 5 / 4 * eta ** 2) * Sg
    f = np.zeros(8)
    f[0] = 1.0
    f[2] = -1247 / 336 - 35 / 12 * eta
    f[3] = 4 * pi - 4 * S - 5 / 4 * d * Sg
    f[4] = -44711 / 9072 + 9271 / 504 * eta + 65 / 18 * eta ** 2
    f[5] = (-9 / 2 + 272 / 9 * eta) * S + (-13 / 16 + 43 / 4 * eta) * d * Sg
    f[6] = -16 * pi * S - 31 / 6 * pi * d * Sg
    f[7] = ((476645 / 6804 + 6172 / 189 * eta - 2810 / 27 * eta ** 2) * S
            + (9535 / 336 + 1849 / 126 * eta - 1501 / 36 * eta ** 2) * d * Sg)
    num = np.array([(k + 2) / 2 * e[k] for k in range(8)])  # E'(v) / (-eta v)
    a = np.zeros(8)
    for k in range(8):                                       # series quotient num / f
        a[k] = num[k] - sum(f[j] * a[k - j] for j in range(1, k + 1))
    phi = {k: 40 * a[k] / ((k - 8) * (k - 5)) for k in (2, 3, 4, 6, 7)}
    return phi, -40 / 3 * a[5]


def test_energy_flux_derivation_reproduces_published_nonspinning_terms():
    """The stationary-phase derivation from the energy and the flux, at zero spin, gives the
    published 1PN, 1.5PN and 2PN phase coefficients: this checks the derivation that the next
    test uses on the spin-orbit terms."""
    for q in (1.0, 0.6, 0.2):
        eta = q / (1 + q) ** 2
        phi, l5 = _taylorf2_from_energy_and_flux(q, 0.0, 0.0)
        assert phi[2] == pytest.approx(3715 / 756 + 55 * eta / 9, rel=1e-13)
        assert phi[3] == pytest.approx(-16 * math.pi, rel=1e-13)
        assert phi[4] == pytest.approx(15293365 / 508032 + 27145 * eta / 504 + 3085 * eta ** 2 / 72, rel=1e-13)


@pytest.mark.parametrize("q", [1.0, 0.7, 0.25])
def test_spin_orbit_phase_terms_follow_from_energy_and_flux(q):
    """Every spin-orbit term of the oracle's phase -- 1.5PN, the 2.5PN v^5 ln v term, 3PN and
    3.5PN -- equals the one derived from the published spin-orbit energy and flux
    (`_taylorf2_from_energy_and_flux`), for each spin separately.  The part linear in one spin
    is taken by a central difference, which removes the spin-spin term, and is exactly a
    combination of v^3, v^5, v^5 ln v, v^6 and v^7 in Psi * 128 eta v^5 / 3; a least-squares
    fit recovers each coefficient.  The constant v^5 coefficient is a constant phase (absorbed
    in the coalescence phase) and is not compared."""
    mc, h = 1.2, 0.5
    eta = q / (1 + q) ** 2
    M = mc * eta ** -0.6 * TSUN
    v = np.linspace(0.05, 0.4, 40)
    f = v ** 3 / (math.pi * M)
    A = np.stack([v ** 3, v ** 5, v ** 5 * np.log(v), v ** 6, v ** 7], axis=1)
    scale = np.abs(A).max(axis=0)
    for spin in ((h, 0.0), (0.0, h)):
        neg = (-spin[0], -spin[1])
        g = np.array([oracle.pn_psi(mc, q, *spin, fi) - oracle.pn_psi(mc, q, *neg, fi) for fi in f])
        g *= 128 * eta * v ** 5 / 3 / (2 * h)
        coef = np.linalg.lstsq(A / scale, g, rcond=None)[0] / scale
        pp, lp = _taylorf2_from_energy_and_flux(q, *spin)
        pm, lm = _taylorf2_from_energy_and_flux(q, *neg)
        lin = {k: (pp[k] - pm[k]) / (2 * h) for k in (3, 6, 7)}
        derived = [lin[3], (lp - lm) / (2 * h), lin[6], lin[7]]
        assert [coef[0], coef[2], coef[3], coef[4]] == pytest.approx(derived, rel=1e-10)


def test_chirp_time_newtonian():
    """t(f) = (1/2pi) dPsi/df -> -(5/256) Mc (pi Mc f)^(-8/3) at low v (textbook chirp time)."""
    mc, q = 30.0, 0.9
    eta = q / (1 + q) ** 2
    M = mc * eta ** -0.6 * TSUN
    v = 1e-3
    f = v ** 3 / (math.pi * M)
    h = f * 1e-6
    dpsi = (oracle.pn_psi(mc, q, 0, 0, f + h) - oracle.pn_psi(mc, q, 0, 0, f - h)) / (2 * h)
    mcs = mc * TSUN
    assert dpsi / (2 * math.pi) == pytest.approx(-(5 / 256) * mcs * (math.pi * mcs * f) ** (-8 / 3), rel=1e-4)


def test_equal_mass_swap_symmetry():
    """q = 1: swapping the spins leaves the phase unchanged (delta = 0)."""
    a = oracle.pn_psi(25.0, 1.0, 0.3, -0.6, 40.0)
    b = oracle.pn_psi(25.0, 1.0, -0.6, 0.3, 40.0)
    assert a == pytest.approx(b, rel=1e-14)


# ---------------------------------------------------------------- detector response
def test_antenna_pattern_pole_textbook():
    """Detector at the north pole, arms on x and y: textbook
    F+ = 1/2 (1 + cos^2 th) cos 2ph cos 2psi - cos th sin 2ph sin 2psi,
    Fx = 1/2 (1 + cos^2 th) cos 2ph sin 2psi + cos th sin 2ph cos 2psi.
    The wave-frame basis used here (e_N = -e_theta) gives F+ = -F+(textbook), Fx = Fx(textbook);
    F+^2 + Fx^2 is psi-independent; the delay is -R sin(dec)/c."""
    g = I.pole_geometry()[None]
    rng = np.random.default_rng(3)
    for _ in range(20):
        th, ph, psi = rng.uniform(0, math.pi), rng.uniform(0, 2 * math.pi), rng.uniform(0, math.pi)
        gmst = 0.4
        out = oracle.antenna(g, gmst, psi, ph + gmst, math.pi / 2 - th)[0]
        fp = 0.5 * (1 + math.cos(th) ** 2) * math.cos(2 * ph) * math.cos(2 * psi) - math.cos(th) * math.sin(2 * ph) * math.sin(2 * psi)
        fx = 0.5 * (1 + math.cos(th) ** 2) * math.cos(2 * ph) * math.sin(2 * psi) + math.cos(th) * math.sin(2 * ph) * math.cos(2 * psi)
        assert out[0] == pytest.approx(-fp, abs=1e-13)
        assert out[1] == pytest.approx(fx, abs=1e-13)
        assert out[2] == pytest.approx(-I.R_EARTH * math.cos(th) / 299792458.0, rel=1e-13)
        o2 = oracle.antenna(g, gmst, psi + 0.7, ph + gmst, math.pi / 2 - th)[0]
        assert o2[0] ** 2 + o2[1] ** 2 == pytest.approx(out[0] ** 2 + out[1] ** 2, rel=1e-12)


# ---------------------------------------------------------------- brute force (mpmath)
def test_tiny_grid_against_mpmath_50_digits():
    """A 12-bin, 2-detector case at long-segment phases (f up to 2048 Hz, t_ref = 126 s)
    recomputed in 50-digit arithmetic: the FP64 oracle agrees to 1e-9 relative."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    rng = np.random.default_rng(5)
    freqs = 2030.0 + np.arange(12) / 128.0
    geom = np.stack([I.site_geometry(*I.SITES["H"]), I.site_geometry(*I.SITES["V"])])
    psd = np.tile(I.psd_aligo(freqs), (2, 1))
    th = np.array([1.2, 0.85, 0.02, -0.03, 40.0, 0.7, 1.1, 2.5, -0.4, 0.013, 0.8])
    skel = I.Event("tiny", freqs, np.zeros((2, 12), complex), psd, geom, 1.7, 126.0, 1, 128.0, th, 0.0, None)
    h = oracle.waveform(skel, th)
    d = h * (1 + 0.3 * rng.standard_normal(h.shape)) + 1e-24 * rng.standard_normal(h.shape)
    ev = skel.with_strain(d)
    th_t = th.copy()
    th_t[0] = 1.2000003
    got = oracle.loglike(ev, th_t[None])[0]

    m = mp.mpf
    pi = mp.pi
    mc, q, c1_, c2_, dl, iota, psi, ra, dec, tc, phic = [m(float(x)) for x in th_t]
    eta = q / (1 + q) ** 2
    delta = (1 - q) / (1 + q)
    m1, m2 = 1 / (1 + q), q / (1 + q)
    chis, chia = (c1_ + c2_) / 2, (c1_ - c2_) / 2
    Ms = mc * eta ** m("-0.6") * m("4.925490947e-6")
    g = m(0.5772156649015329)
    p2 = m(20) / 9 * (m(743) / 336 + m(11) / 4 * eta)
    beta = (m(113) / 12 * m1 ** 2 + m(25) / 4 * eta) * c1_ + (m(113) / 12 * m2 ** 2 + m(25) / 4 * eta) * c2_
    p3 = -16 * pi + 4 * beta
    p4 = 10 * (m(3058673) / 1016064 + m(5429) / 1008 * eta + m(617) / 144 * eta ** 2) - 10 * m(79) / 8 * eta * c1_ * c2_
    gam = (m(732985) / 2268 - m(24260) / 81 * eta - m(340) / 9 * eta ** 2) * chis + (m(732985) / 2268 + m(140) / 9 * eta) * delta * chia
    p5c = pi * (m(38645) / 756 - m(65) / 9 * eta) - gam
    p6c = (m(11583231236531) / 4694215680 - m(640) / 3 * pi ** 2 - m(6848) / 21 * g
           + eta * (m(-15737765635) / 3048192 + m(2255) / 12 * pi ** 2) + m(76055) / 1728 * eta ** 2
           - m(127825) / 1296 * eta ** 3 + pi * (m(2270) / 3 * delta * chia + (m(2270) / 3 - 520 * eta) * chis))
    p7 = (pi * (m(77096675) / 254016 + m(378515) / 1512 * eta - m(74045) / 756 * eta ** 2)
          + (m(-25150083775) / 3048192 + m(10566655595) / 762048 * eta - m(1042165) / 3024 * eta ** 2 + m(5345) / 36 * eta ** 3) * chis
          + delta * (m(-25150083775) / 3048192 + m(26804935) / 6048 * eta - m(1985) / 48 * eta ** 2) * chia)
    amp = mp.sqrt(m(5) / 24) * pi ** (m(-2) / 3) * (mc * m("4.925490947e-6")) ** (m(5) / 6) * m(299792458) / (dl * m("3.085677581491367e22"))
    vlso = 1 / mp.sqrt(6)
    total = m(0)
    df = m(1) / 128
    for dd in range(2):
        gv = [m(float(x)) for x in geom[dd]]
        lam = ra - m(1.7)
        n = [mp.cos(dec) * mp.cos(lam), mp.cos(dec) * mp.sin(lam), mp.sin(dec)]
        eE = [-mp.sin(lam), mp.cos(lam), m(0)]
        eN = [-mp.sin(dec) * mp.cos(lam), -mp.sin(dec) * mp.sin(lam), mp.cos(dec)]
        X = [mp.cos(psi) * eE[i] + mp.sin(psi) * eN[i] for i in range(3)]
        Y = [-mp.sin(psi) * eE[i] + mp.cos(psi) * eN[i] for i in range(3)]
        xa, ya = gv[3:6], gv[6:9]
        Fp = sum(m(0.5) * (xa[i] * xa[k] - ya[i] * ya[k]) * (X[i] * X[k] - Y[i] * Y[k]) for i in range(3) for k in range(3))
        Fx = sum(m(0.5) * (xa[i] * xa[k] - ya[i] * ya[k]) * (X[i] * Y[k] + Y[i] * X[k]) for i in range(3) for k in range(3))
        dt = -(gv[0] * n[0] + gv[1] * n[1] + gv[2] * n[2]) / m(299792458)
        for j in range(12):
            f = m(float(freqs[j]))
            v = mp.cbrt(pi * Ms * f)
            ser = (1 + p2 * v ** 2 + p3 * v ** 3 + p4 * v ** 4 + p5c * (1 + 3 * mp.log(v / vlso)) * v ** 5
                   + (p6c - m(6848) / 21 * mp.log(4 * v)) * v ** 6 + p7 * v ** 7)
            Psi = 2 * pi * f * (m(126) + tc + dt) - phic - pi / 4 + 3 / (128 * eta * v ** 5) * ser
            a = amp * f ** (m(-7) / 6)
            pr = Fp * (1 + mp.cos(iota) ** 2) / 2
            pim = -Fx * mp.cos(iota)
            hr = a * (pr * mp.cos(Psi) + pim * mp.sin(Psi))
            hi = a * (pim * mp.cos(Psi) - pr * mp.sin(Psi))
            w = 4 * df / m(float(psd[dd, j]))
            dr, di = m(float(d[dd, j].real)), m(float(d[dd, j].imag))
            total += w * (dr * hr + di * hi - (hr ** 2 + hi ** 2) / 2)
    assert got == pytest.approx(float(total), rel=1e-9, abs=1e-12)


# ---------------------------------------------------------------- gradient
def test_dual_gradient_matches_central_differences(c2):
    """Dual-number gradient vs central finite differences (h = 1e-6 relative, ISCO bin fixed)."""
    rng = np.random.default_rng(7)
    th = I.proposals(c2, 6, 3)
    l, g = oracle.grad(c2, th)
    assert np.allclose(l, oracle.loglike(c2, th), rtol=1e-13, atol=1e-10)
    for b in range(th.shape[0]):
        for k in range(11):
            hstep = 1e-6 * max(abs(th[b, k]), 1e-2)
            tp, tm = th[b].copy(), th[b].copy()
            tp[k] += hstep
            tm[k] -= hstep
            if k in (0, 1):  # mass moves the ISCO bin: skip points where the cut changes
                def ncut(t):
                    eta = t[1] / (1 + t[1]) ** 2
                    fi = 1 / (6 ** 1.5 * math.pi * t[0] * eta ** -0.6 * TSUN)
                    return np.searchsorted(c2.freqs, fi, side="right")
                if ncut(tp) != ncut(tm):
                    continue
            fd = (oracle.loglike(c2, tp[None])[0] - oracle.loglike(c2, tm[None])[0]) / (2 * hstep)
            scale = max(1.0, abs(g[b, k]))
            assert abs(fd - g[b, k]) < 2e-4 * scale, (b, k, fd, g[b, k])


# ---------------------------------------------------------------- prior transform
def test_prior_transform_distributions(c2):
    """Each unit-cube map reproduces its analytic CDF (Kolmogorov-Smirnov)."""
    smp = c2.sampling
    u = np.random.default_rng(9).uniform(0, 1, (4000, smp.D))
    th = oracle.prior_transform(smp, u)
    lo, hi = smp.lo[4], smp.hi[4]
    assert stats.kstest(th[:, 4], lambda x: (x ** 3 - lo ** 3) / (hi ** 3 - lo ** 3)).pvalue > 1e-3
    assert stats.kstest(th[:, 5], lambda x: (1 - np.cos(x)) / 2).pvalue > 1e-3
    assert stats.kstest(th[:, 8], lambda x: (1 + np.sin(x)) / 2).pvalue > 1e-3
    assert stats.kstest(th[:, 0], "uniform", args=(smp.lo[0], smp.hi[0] - smp.lo[0])).pvalue > 1e-3


# ---------------------------------------------------------------- random numbers
def philox_kat():
    """The published known-answer vectors of Philox4x32-10 (tests/golden/philox4x32_10_kat.json)."""
    kat = json.load(open(os.path.join(HERE, "golden", "philox4x32_10_kat.json")))
    return [([int(x, 16) for x in v["counter"]], [int(x, 16) for x in v["key"]], [int(x, 16) for x in v["output"]])
            for v in kat["vectors"]]


def test_philox_known_answers():
    """The oracle's Philox4x32-10 reproduces the generator's published known-answer vectors (Salmon et
    al. 2011): a swapped multiplier, a wrong key schedule or a permuted output word fails."""
    for ctr, key, want in philox_kat():
        got = [int(x) for x in oracle.philox(ctr, key)]
        assert got == want, (ctr, key, [hex(x) for x in got])


def test_philox_uniformity_and_counter_independence():
    """Philox4x32-10 words: uniform (chi^2 on 256 bins), distinct for neighbouring counters,
    and the Box-Muller normals of the walk stream are N(0,1) (KS)."""
    words = np.concatenate([oracle.philox([i, 7, 3, 0], [123, 456]) for i in range(5000)])
    cnt = np.bincount(words >> 24, minlength=256)
    assert stats.chisquare(cnt).pvalue > 1e-4
    a = oracle.philox([0, 0, 0, 0], [1, 0])
    b = oracle.philox([1, 0, 0, 0], [1, 0])
    c = oracle.philox([0, 0, 0, 0], [2, 0])
    assert len({tuple(a), tuple(b), tuple(c)}) == 3
    w = np.stack([oracle.philox([0, s, 5, 0], [99, 0]) for s in range(1, 3001)]).astype(np.float64)
    u1 = (w[:, 0] + 1) * 2.0 ** -32
    u2 = w[:, 1] * 2.0 ** -32
    z = np.sqrt(-2 * np.log(u1)) * np.cos(2 * np.pi * u2)
    assert stats.kstest(z, "norm").pvalue > 1e-3


# ---------------------------------------------------------------- nested sampling
def eq5(n_cores, n_live):
    """Speed-up law of the paper, Eq. 5: S = n_live ln(1 + n_cores / n_live)."""
    return n_live * math.log(1 + n_cores / n_live)


def test_eq5_agrees_with_table1_measurements():
    """The paper's measured GW150914 wall times (Table 1) follow Eq. 5 to within 5%."""
    g = json.load(open(os.path.join(HERE, "golden", "table1_walltimes.json")))
    t = dict(zip(g["cores"], g["walltime_hours"]))
    for a, b in ((16, 64), (16, 640)):
        assert t[a] / t[b] == pytest.approx(eq5(b, g["n_live"]) / eq5(a, g["n_live"]), rel=0.05)


def gauss_box_lnz(D, mu, sigma):
    return sum(math.log(0.5 * (special.erf((1 - m) / (sigma * math.sqrt(2))) - special.erf(-m / (sigma * math.sqrt(2)))))
               for m in mu)


def gauss_box_information(mu, sigma):
    """H = int P ln(L / Z) for the normalised Gaussian L in the unit cube: per coordinate, with the
    truncated normal's standardised bounds a, b and mass Z_i, E[z^2] = 1 - (b phi(b) - a phi(a)) / Z_i
    and H_i = -ln(2 pi sigma^2) / 2 - E[z^2] / 2 - ln Z_i."""
    h = 0.0
    for m in mu:
        a, b = -m / sigma, (1 - m) / sigma
        z = stats.norm.cdf(b) - stats.norm.cdf(a)
        ez2 = 1 - (b * stats.norm.pdf(b) - a * stats.norm.pdf(a)) / z
        h += -0.5 * math.log(2 * math.pi * sigma ** 2) - 0.5 * ez2 - math.log(z)
    return h


@pytest.mark.slow
def test_ns_gaussian_in_box_evidence():
    """Oracle NS recovers lnZ of a Gaussian in the unit cube (closed form with erf) over 8 seeds,
    and its information H (which sets lnZ_err = sqrt(H / K)) the truncated normal's closed form."""
    D, sigma = 3, 0.08
    mu = np.array([0.1, 0.55, 0.9])
    truth = gauss_box_lnz(D, mu, sigma)
    h_true = gauss_box_information(mu, sigma)
    errs, sig, hs = [], [], []
    for s in range(8):
        r = oracle.ns_run_gauss(D, mu, sigma, K=200, n_chains=100, walk_len=25, seed=1000 + s, dlogz=0.05)
        errs.append(r["lnZ"] - truth)
        sig.append(r["lnZ_err"])
        hs.append(r["H"])
        assert abs(r["lnZ"] - truth) < 4 * r["lnZ_err"]
        assert r["lnZ_err"] == pytest.approx(math.sqrt(r["H"] / 200), rel=1e-12)
        assert abs(r["H"] - h_true) < 0.6      # the runs' H scatter by ~0.13 (K = 200)
    assert abs(np.mean(errs)) < 3 * np.mean(sig) / math.sqrt(len(errs)) + 0.02
    assert abs(np.mean(hs) - h_true) < 0.15


@pytest.mark.slow
def test_ns_gaussian_in_box_posterior_moments():
    """The dead points weighted by L_i dX_i / Z (final live points included, Algorithm 1) reproduce the
    truncated normal's mean mu + sigma (phi(a) - phi(b)) / Z_i and standard deviation
    sigma sqrt(1 + (a phi(a) - b phi(b)) / Z_i - ((phi(a) - phi(b)) / Z_i)^2) per coordinate: per run
    within 5 standard errors of the weighted sample (effective size from the weights), and over 8
    runs within 4."""
    D, sigma = 3, 0.08
    mu = np.array([0.1, 0.55, 0.9])
    a, b = -mu / sigma, (1 - mu) / sigma
    z = stats.norm.cdf(b) - stats.norm.cdf(a)
    pa, pb = stats.norm.pdf(a), stats.norm.pdf(b)
    mean_t = mu + sigma * (pa - pb) / z
    sd_t = sigma * np.sqrt(1 + (a * pa - b * pb) / z - ((pa - pb) / z) ** 2)
    means, sds, ess_all = [], [], []
    for s in range(8):
        r = oracle.ns_run_gauss(D, mu, sigma, K=200, n_chains=100, walk_len=25, seed=1000 + s, dlogz=0.05,
                                max_dead=100000)
        assert len(r["dead_lnl"]) == r["n_dead"]
        w = np.exp(r["dead_lnl"] + r["dead_logwt"] - r["lnZ"])
        assert w.sum() == pytest.approx(1.0, rel=1e-12)
        u = r["dead_u"]
        m = (w[:, None] * u).sum(0)
        sd = np.sqrt((w[:, None] * (u - m) ** 2).sum(0))
        ess = 1.0 / (w ** 2).sum()
        assert np.all(np.abs(m - mean_t) < 5 * sd_t / math.sqrt(ess))
        assert np.all(np.abs(sd / sd_t - 1) < 5 / math.sqrt(2 * ess))
        means.append(m)
        sds.append(sd)
        ess_all.append(ess)
    n_eff = len(means) * np.mean(ess_all)
    assert np.all(np.abs(np.mean(means, 0) - mean_t) < 4 * sd_t / math.sqrt(n_eff))
    assert np.all(np.abs(np.mean(sds, 0) / sd_t - 1) < 4 / math.sqrt(2 * n_eff))


@pytest.mark.slow
def test_ns_consumption_follows_eq5():
    """Mean candidates consumed per round ~ K ln(1 + B/K) (Eq. 5) for several batch sizes."""
    D, sigma = 2, 0.1
    mu = np.array([0.5, 0.5])
    K = 200
    for B in (50, 200, 800):
        r = oracle.ns_run_gauss(D, mu, sigma, K=K, n_chains=B, walk_len=30, seed=77 + B, dlogz=0.05)
        assert r["consumed_per_round"] == pytest.approx(eq5(B, K), rel=0.08)


@pytest.mark.slow
def test_ns_gw_c1_recovers_injection(c1):
    """Oracle NS on the 1-detector zero-noise event: finite lnZ and lnZ_err, the posterior mean of
    Mc within 0.05 Msun of the injection (SNR 20)."""
    r = oracle.ns_run(c1, c1.sampling, K=150, n_chains=150, walk_len=20, seed=5, dlogz=0.1, max_dead=20000)
    assert np.isfinite(r["lnZ"]) and 0 < r["lnZ_err"] < 1
    w = np.exp(r["dead_lnl"] + r["dead_logwt"] - r["lnZ"])
    th = oracle.prior_transform(c1.sampling, r["dead_u"])
    assert abs(np.sum(w * th[:, 0]) / np.sum(w) - 10.0) < 0.05


def test_ns_replace_semantics(c1):
    """Walk outputs: n_acc in [0, walk_len]; chains that never moved return their start point;
    every moved chain ends at lnL >= L* and its lnL re-evaluates exactly; no chain starts at the worst;
    a fixed (seed, counter) reproduces the result."""
    smp = c1.sampling
    rng = np.random.default_rng(2)
    K = 64
    u = rng.uniform(0, 1, (K, smp.D))
    ll = oracle.loglike(c1, oracle.prior_transform(smp, u))
    worst = int(np.argmin(ll))
    chol = np.diag([0.05] * smp.D)
    out = oracle.ns_replace(c1, smp, u, ll, worst, ll[worst], 42, 3, 96, 10, 1.0, chol)
    ou, ol, on, st = out
    assert np.all((on >= 0) & (on <= 10))
    assert np.all(st != worst)
    moved = on > 0
    assert np.all(ol[moved] >= ll[worst])
    assert np.allclose(ou[~moved], u[st[~moved]]) and np.allclose(ol[~moved], ll[st[~moved]])
    assert np.array_equal(oracle.loglike(c1, oracle.prior_transform(smp, ou)), ol)
    out2 = oracle.ns_replace(c1, smp, u, ll, worst, ll[worst], 42, 3, 96, 10, 1.0, chol)
    assert all(np.array_equal(a, b) for a, b in zip(out, out2))



# ---------------------------------------------------------------- calibration model
def _cal_theta(ev, th11, dA, dphi):
    """Row [11 + 2 n_nodes n_det] from per-detector node arrays dA, dphi [n_det, n_nodes]."""
    n_det = ev.geom.shape[0]
    cal = np.concatenate([np.concatenate([dA[d], dphi[d]]) for d in range(n_det)])
    return np.concatenate([th11, cal])


def test_cal_spline_is_scipy_natural_cubic_spline():
    """The oracle's spline equals scipy's natural CubicSpline, inside and outside the nodes."""
    from scipy.interpolate import CubicSpline
    rng = np.random.default_rng(5)
    for n in (2, 3, 4, 10, 16):
        x = np.sort(rng.uniform(2.5, 7.5, n))
        x[1:] = np.maximum(x[1:], x[:-1] + 0.05)
        y = rng.normal(size=n)
        q = np.linspace(x[0] - 0.7, x[-1] + 0.7, 777)
        ref = CubicSpline(x, y, bc_type="natural")(q)
        assert np.abs(oracle.cal_spline(x, y, q) - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())


def test_cal_zero_corrections_reduce_to_uncalibrated(c2):
    nodes = I.cal_node_freqs(20.0, 1024.0)
    th = I.proposals(c2, 8, 3)
    rows = np.stack([_cal_theta(c2, t, np.zeros((3, 10)), np.zeros((3, 10))) for t in th])
    np.testing.assert_allclose(oracle.loglike_cal(c2, nodes, rows), oracle.loglike(c2, th), rtol=1e-13, atol=1e-12)


def test_cal_constant_amplitude_is_a_distance_rescale(c2):
    """dA = a at every node: C h = (1 + a) h, the template of distance d_L / (1 + a)."""
    nodes = I.cal_node_freqs(20.0, 1024.0)
    th = I.proposals(c2, 6, 4)
    for a in (-0.2, 0.07, 0.3):
        rows = np.stack([_cal_theta(c2, t, np.full((3, 10), a), np.zeros((3, 10))) for t in th])
        ref_th = th.copy()
        ref_th[:, I.IDX["dl"]] /= 1.0 + a
        np.testing.assert_allclose(oracle.loglike_cal(c2, nodes, rows), oracle.loglike(c2, ref_th),
                                   rtol=1e-11, atol=1e-9)


def test_cal_constant_phase_is_a_coalescence_phase_shift(c2):
    """dphi = p0 at every node: C h = e^{i p0} h, the template with phi_c + p0."""
    nodes = I.cal_node_freqs(20.0, 1024.0)
    th = I.proposals(c2, 6, 5)
    for p0 in (-0.4, 0.15, 1.0):
        rows = np.stack([_cal_theta(c2, t, np.zeros((3, 10)), np.full((3, 10), p0)) for t in th])
        ref_th = th.copy()
        ref_th[:, I.IDX["phic"]] += p0
        np.testing.assert_allclose(oracle.loglike_cal(c2, nodes, rows), oracle.loglike(c2, ref_th),
                                   rtol=1e-11, atol=1e-9)


def test_cal_loglike_brute_force_with_scipy_splines(c2):
    """Different corrections per detector: lnL = <d|C h> - <C h|C h>/2 from the oracle's
    waveform, scipy's natural splines in ln f and a numpy inner product."""
    from scipy.interpolate import CubicSpline
    nodes = I.cal_node_freqs(20.0, 1024.0)
    rng = np.random.default_rng(9)
    th = I.proposals(c2, 4, 6)
    x = np.log(c2.freqs)
    for t in th:
        dA = 0.1 * rng.standard_normal((3, 10))
        dphi = 0.1 * rng.standard_normal((3, 10))
        h = oracle.waveform(c2, t)
        C = np.stack([(1.0 + CubicSpline(np.log(nodes), dA[d], bc_type="natural")(x))
                      * np.exp(1j * CubicSpline(np.log(nodes), dphi[d], bc_type="natural")(x)) for d in range(3)])
        ch = C * h
        ref = inner(c2, c2.strain, ch) - 0.5 * inner(c2, ch, ch)
        got = oracle.loglike_cal(c2, nodes, _cal_theta(c2, t, dA, dphi)[None])[0]
        assert got == pytest.approx(ref, rel=1e-10, abs=1e-8)


def test_cal_gradient_matches_central_differences(c2):
    """Gradient of the calibrated lnL by dual numbers over all 11 + 60 parameters against central
    differences of the calibrated lnL (h = 1e-6 relative for the source parameters, 1e-5 for the
    node values; points where a mass step moves the ISCO bin are skipped)."""
    nodes = I.cal_node_freqs(20.0, 1024.0)
    th = I.calibrated_proposals(c2, 3, 12)
    lnl, g = oracle.grad_cal(c2, nodes, th)
    assert np.allclose(lnl, oracle.loglike_cal(c2, nodes, th), rtol=1e-13, atol=1e-10)
    D = th.shape[1]

    def ncut(t):
        eta = t[1] / (1 + t[1]) ** 2
        fi = 1 / (6 ** 1.5 * math.pi * t[0] * eta ** -0.6 * TSUN)
        return np.searchsorted(c2.freqs, fi, side="right")

    rows, idx, steps = [], [], []
    for b in range(th.shape[0]):
        for k in range(D):
            hstep = 1e-6 * max(abs(th[b, k]), 1e-2) if k < 11 else 1e-5
            tp, tm = th[b].copy(), th[b].copy()
            tp[k] += hstep
            tm[k] -= hstep
            if k in (0, 1) and ncut(tp) != ncut(tm):
                continue
            rows += [tp, tm]
            idx.append((b, k))
            steps.append(hstep)
    vals = oracle.loglike_cal(c2, nodes, np.array(rows)).reshape(-1, 2)
    for (b, k), hstep, (lp, lm) in zip(idx, steps, vals):
        fd = (lp - lm) / (2 * hstep)
        assert abs(fd - g[b, k]) < 2e-4 * max(1.0, abs(g[b, k])), (b, k, fd, g[b, k])


def test_cal_gradient_at_zero_corrections_closed_form(c2):
    """With every correction zero, C = 1 and the node derivatives have closed forms in the cardinal
    natural splines s_k (scipy, through the k-th unit vector, in ln f):
      d lnL / d dA_d,k   = sum_j s_k(ln f_j) w_j [Re(conj(d_j) h_j) - |h_j|^2],
      d lnL / d dphi_d,k = sum_j s_k(ln f_j) w_j Re(conj(d_j) i h_j),   w_j = 4 df / S_j,
    with h the oracle's (pinned) waveform; the source derivatives are the uncalibrated gradient."""
    from scipy.interpolate import CubicSpline
    nodes = I.cal_node_freqs(20.0, 1024.0)
    nn = nodes.size
    x = np.log(c2.freqs)
    s = np.stack([CubicSpline(np.log(nodes), np.eye(nn)[k], bc_type="natural")(x) for k in range(nn)])
    w = 4.0 * c2.df / c2.psd
    for t in I.proposals(c2, 2, 13):
        zero = np.zeros((3, nn))
        _, g = oracle.grad_cal(c2, nodes, _cal_theta(c2, t, zero, zero)[None])
        _, g0 = oracle.grad(c2, t[None])
        assert np.allclose(g[0, :11], g0[0], rtol=1e-10, atol=1e-9)
        h = oracle.waveform(c2, t)
        for d in range(3):
            ta = w[d] * (np.real(np.conj(c2.strain[d]) * h[d]) - np.abs(h[d]) ** 2)
            tp = w[d] * np.real(np.conj(c2.strain[d]) * 1j * h[d])
            got = g[0, 11 + 2 * nn * d: 11 + 2 * nn * (d + 1)]
            ref = np.concatenate([s @ ta, s @ tp])
            assert np.allclose(got, ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max()), (d, got, ref)


def test_inverse_normal_cdf_is_scipy_ndtri():
    """The oracle's Phi^{-1} (calibration priors) equals scipy's ndtri from the far tails to the centre."""
    u = np.concatenate([np.geomspace(1e-300, 0.5, 400), 1.0 - np.geomspace(1e-16, 0.5, 400),
                        np.random.default_rng(0).uniform(size=2000)])
    got, ref = oracle.inv_normal_cdf(u), special.ndtri(u)
    assert np.all(np.abs(got - ref) <= 2e-15 * np.maximum(1.0, np.abs(ref)))
    nz = np.abs(ref) > 1e-3
    assert np.all(np.abs(got[nz] - ref[nz]) <= 4e-15 * np.abs(ref[nz]))
    assert list(oracle.inv_normal_cdf([0.0, 0.5, 1.0])) == [-np.inf, 0.0, np.inf]


@pytest.mark.slow
def test_ns_with_vanishing_calibration_priors_reproduces_lnz(c1):
    """Calibrated NS whose calibration priors are 1e-9 wide (8 extra walk coordinates that change no
    likelihood) gives the uncalibrated evidence within the sampling error."""
    nodes = np.geomspace(20.0, 512.0, 4)
    kw = dict(K=150, n_chains=150, walk_len=20, dlogz=0.1)
    ref = oracle.ns_run(c1, c1.sampling, seed=5, **kw)
    got = oracle.ns_run_cal(c1, c1.sampling, (nodes, 1e-9, 1e-9), seed=6, **kw)
    sig = math.hypot(ref["lnZ_err"], got["lnZ_err"])
    assert abs(got["lnZ"] - ref["lnZ"]) < 4 * sig, (got, ref)
