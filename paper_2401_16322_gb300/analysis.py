"""Dispersion and dissipation of the time integrators (the analysis of Sec. 4).

For the undamped semi-discrete system an eigenmode of frequency omega (eigenvalue i omega of
H) advances by exp(i omega dt) per step.  A one-step integrator multiplies it by its
amplification factor R(i omega dt) instead:

* Faber: R = sum_j a_j F_j(i omega), with Sec. 3.2's recurrence and the coefficients of
  exp(dt z) on the ellipse (gamma, c0, c1), computed here by the trapezoid rule on
  N = max(4m, 64) nodes, as the library does;
* HORK(m): the degree-m Taylor polynomial of exp (it is m-th order linear RK);
* RK4-4: the degree-4 Taylor polynomial; RK3-2 as printed: 1 + z + z^2/2 + z^3/4;
* leap-frog: the principal root of zeta^2 - (2 + z^2) zeta + 1 = 0 (the two-step scheme on
  u_tt = -omega^2 u); |zeta| = 1 for omega dt <= 2.

Krylov has no fixed amplification function: its polynomial depends on the state.  It is
exact on the span of its basis.

Dissipation is |R| - 1 and dispersion the relative phase error arg(R) / (omega dt) - 1.  Both
vanish for the exact exponential.  This is host-side analysis of the methods; it is not part
of the GPU path.

``trace_errors`` is the paper's own measure (Sec. 4.1), taken on recorded traces instead of
amplification factors: with F_ref and F_appr the discrete Fourier transforms of a reference
and an approximate receiver trace, F_ref = exp(k + i l) F_appr defines k(omega) (dissipation)
and l(omega) (dispersion), and the two errors are the means of |k| and |l| over the
frequencies where |F_ref| or |F_appr| exceeds 1 % of max |F_ref|.
"""
import math

import numpy as np


def faber_coefficients(dt, gamma, c0, c1, m, nodes=None):
    """a_j = (1/N) sum_k exp(dt psi(w_k)) w_k^-j, psi(w) = gamma (w + c0 + c1 / w), w_k on the
    unit circle (trapezoid rule, exponentially convergent)."""
    n = max(4 * m, 64) if nodes is None else nodes
    w = np.exp(2j * np.pi * np.arange(n) / n)
    f = np.exp(dt * gamma * (w + c0 + c1 / w))
    return np.array([(np.sum(f * w ** (-j)) / n).real for j in range(m + 1)])


def amplification(method, m, omega, dt, ellipse=None):
    """R(i omega dt) of ``method`` (faber needs ``ellipse`` = (gamma, c0, c1)).  A complex
    omega = lambda / i evaluates R at z = lambda dt for an eigenvalue lambda with damping."""
    omega = np.asarray(omega)
    omega = omega.astype(np.complex128 if np.iscomplexobj(omega) else np.float64)
    z = 1j * omega * dt
    if method in ("hork", "hork-horner"):      # the same polynomial, either evaluation order
        out, term = np.ones_like(z), np.ones_like(z)
        for k in range(1, m + 1):
            term = term * z / k
            out = out + term
        return out
    if method == "rk44":
        return amplification("hork", 4, omega, dt)
    if method == "rk32":
        return 1 + z + z ** 2 / 2 + z ** 3 / 4
    if method in ("leapfrog", "leapfrog-difference"):      # one scheme, two storage forms
        b = 1 + z ** 2 / 2
        root = np.sqrt(b * b - 1 + 0j)
        z1, z2 = b + root, b - root
        # omega dt <= 2: both roots on the unit circle, the principal one with positive phase
        # (it tends to 1 as omega dt -> 0); beyond 2 the larger root (the growing mode)
        a1, a2 = np.abs(z1), np.abs(z2)
        on_circle = np.abs(a1 - a2) < 1e-12
        return np.where(on_circle, np.where(np.angle(z1) >= 0, z1, z2), np.where(a1 > a2, z1, z2))
    if method == "faber":
        gamma, c0, c1 = ellipse
        a = faber_coefficients(dt, gamma, c0, c1, m)
        lam = 1j * np.asarray(omega, dtype=np.float64)
        F0, F1 = np.ones_like(lam), lam / gamma - c0
        out = a[0] * F0 + (a[1] * F1 if m >= 1 else 0)
        Fm2, Fm1 = F0, F1
        for j in range(2, m + 1):
            cj = 2 * c1 if j == 2 else c1
            Fj = F1 * Fm1 - cj * Fm2
            out = out + a[j] * Fj
            Fm2, Fm1 = Fm1, Fj
        return out
    raise ValueError(method)


def dispersion_dissipation(method, m, dt, omega_max, ellipse=None, n=2001):
    """Largest |dissipation| and |dispersion| over 0 < omega <= omega_max."""
    om = np.linspace(omega_max / n, omega_max, n)
    R = amplification(method, m, om, dt, ellipse)
    diss = np.abs(R) - 1.0
    disp = np.unwrap(np.angle(R)) / (om * dt) - 1.0      # phase followed past pi
    return float(np.max(np.abs(diss))), float(np.max(np.abs(disp)))


def report(candidates, f_peak, omega_spectrum, ellipse):
    """Dissipation and dispersion of each (method, m, dt) in the source band
    (omega <= 2 pi * 2.5 f_peak) and over the whole spectrum (omega <= omega_spectrum)."""
    band = 2 * math.pi * 2.5 * f_peak
    out = []
    for method, m, dt in candidates:
        if method == "krylov":
            continue
        db, pb = dispersion_dissipation(method, m, dt, band, ellipse)
        ds, ps = dispersion_dissipation(method, m, dt, omega_spectrum, ellipse)
        out.append({"method": method, "m": m, "dt_ms": dt * 1e3,
                    "band_dissipation": db, "band_dispersion": pb,
                    "spectrum_dissipation": ds, "spectrum_dispersion": ps})
    return out


def trace_errors(ref, appr, threshold=0.01):
    """(dissipation, dispersion) of trace ``appr`` against ``ref`` by Sec. 4.1's Fourier measure.

    Readings of what the paper leaves open: the transform is the real DFT of the traces as
    sampled (same length and spacing; the sample spacing scales omega only and cancels);
    "reference or approximated" is the union of the two amplitude tests; l is the principal
    value of arg(F_ref / F_appr), which is the phase error itself while it stays below pi, as
    it does for the small errors the measure is meant for.  A selected bin with F_appr = 0
    gives an infinite dissipation error."""
    ref = np.asarray(ref, dtype=np.float64)
    appr = np.asarray(appr, dtype=np.float64)
    if ref.shape != appr.shape or ref.ndim != 1:
        raise ValueError("traces must be 1-D and of equal length")
    Fr, Fa = np.fft.rfft(ref), np.fft.rfft(appr)
    peak = float(np.max(np.abs(Fr)))
    if peak == 0.0:
        raise ValueError("the reference trace is zero")
    sel = (np.abs(Fr) > threshold * peak) | (np.abs(Fa) > threshold * peak)
    with np.errstate(divide="ignore", invalid="ignore"):
        ratio = Fr[sel] / Fa[sel]
        k = np.where(Fa[sel] == 0, np.inf, np.log(np.abs(ratio)))
        l = np.where(Fa[sel] == 0, 0.0, np.angle(ratio))
    return float(np.mean(np.abs(k))), float(np.mean(np.abs(l)))
