"""Mie series for scattering of a plane wave by a constant-contrast disk (2D) and ball (3D).

TEST INFRASTRUCTURE ONLY: an independent closed-form solution of eq. (helm) used to pin the
whole discrete solve of the oracle (Sec. 1, eq. helm / eq. ls; the paper itself prints no
such check).

Medium: m = m0 inside the disk |x - c| < R, 0 outside, so the wavenumber is
k1 = omega sqrt(1 - m0) inside and k0 = omega outside.  Incident field exp(i omega x_1)
= exp(i omega c_1) sum_n i^n J_n(k0 r) e^{i n theta}.  Continuity of the total field and of
its radial derivative at r = R gives, per angular index n,
    scattered outside:  c_n H_n(k0 r)
    total inside:       a_n J_n(k1 r)
    c_n = i^n [k1 J_n'(k1R) J_n(k0R) - k0 J_n'(k0R) J_n(k1R)]
              / [k0 H_n'(k0R) J_n(k1R) - k1 J_n'(k1R) H_n(k0R)]
    a_n = (i^n J_n(k0R) + c_n H_n(k0R)) / J_n(k1R)
"""

from __future__ import annotations

import numpy as np
import scipy.special as sp


def mie_disk_scattered(X1, X2, omega: float, m0: float, R: float, centre=(0.5, 0.5), nmax=None):
    """Scattered field u (total minus incident, the unknown of eq. ls) at points (X1, X2)."""
    k0 = omega
    k1 = omega * np.sqrt(1.0 - m0)
    if nmax is None:
        nmax = int(k1 * R + 4.0 * (k1 * R) ** (1.0 / 3.0) + 20)
    dx = X1 - centre[0]
    dy = X2 - centre[1]
    r = np.hypot(dx, dy)
    th = np.arctan2(dy, dx)
    inside = r < R
    u = np.zeros(np.shape(X1), dtype=np.complex128)
    pref = np.exp(1j * omega * centre[0])
    for n in range(-nmax, nmax + 1):
        jn0, jn1 = sp.jv(n, k0 * R), sp.jv(n, k1 * R)
        djn0, djn1 = sp.jvp(n, k0 * R), sp.jvp(n, k1 * R)
        hn0, dhn0 = sp.hankel1(n, k0 * R), sp.h1vp(n, k0 * R)
        inn = 1j ** (n % 4)
        cn = inn * (k1 * djn1 * jn0 - k0 * djn0 * jn1) / (k0 * dhn0 * jn1 - k1 * djn1 * hn0)
        an = (inn * jn0 + cn * hn0) / jn1
        e = np.exp(1j * n * th)
        out = cn * sp.hankel1(n, k0 * r[~inside]) * e[~inside]
        u[~inside] += pref * out
        inn_field = an * sp.jv(n, k1 * r[inside]) - inn * sp.jv(n, k0 * r[inside])
        u[inside] += pref * inn_field * e[inside]
    return u


def mie_disk_far_field(theta, omega: float, m0: float, R: float, centre=(0.5, 0.5), nmax=None):
    """Far-field pattern of the scattered field of the same disk, in the convention
    u_s(x) ~ e^{i omega |x|} |x|^{-1/2} u_inf(theta) as |x| -> infinity in direction theta.

    Outside the disk u_s = pref sum_n c_n H_n(k0 r) e^{i n phi} with (r, phi) about the centre
    c; with r = |x| - theta . c + o(1) and H_n(z) ~ sqrt(2 / (pi z)) e^{i (z - n pi/2 - pi/4)},
        u_inf(theta) = pref sqrt(2 / (pi omega)) e^{-i pi/4} e^{-i omega theta . c}
                       sum_n c_n (-i)^n e^{i n theta}."""
    theta = np.asarray(theta, dtype=np.float64)
    k0 = omega
    k1 = omega * np.sqrt(1.0 - m0)
    if nmax is None:
        nmax = int(k1 * R + 4.0 * (k1 * R) ** (1.0 / 3.0) + 20)
    pref = np.exp(1j * omega * centre[0])
    s = np.zeros(theta.shape, dtype=np.complex128)
    for n in range(-nmax, nmax + 1):
        jn0, jn1 = sp.jv(n, k0 * R), sp.jv(n, k1 * R)
        djn0, djn1 = sp.jvp(n, k0 * R), sp.jvp(n, k1 * R)
        hn0, dhn0 = sp.hankel1(n, k0 * R), sp.h1vp(n, k0 * R)
        inn = 1j ** (n % 4)
        cn = inn * (k1 * djn1 * jn0 - k0 * djn0 * jn1) / (k0 * dhn0 * jn1 - k1 * djn1 * hn0)
        s += cn * (-1j) ** (n % 4) * np.exp(1j * n * theta)
    phase = np.exp(-1j * omega * (np.cos(theta) * centre[0] + np.sin(theta) * centre[1]))
    return pref * np.sqrt(2.0 / (np.pi * omega)) * np.exp(-1j * np.pi / 4) * phase * s


def mie_sphere_scattered(X1, X2, X3, omega: float, m0: float, R: float, centre=(0.5, 0.5, 0.5), lmax=None):
    """Scattered field of a plane wave exp(i omega x_1) by a constant-contrast ball (3D).

    With cos(theta) = (x_1 - c_1) / r and exp(i k r cos theta) = sum_l (2l+1) i^l j_l(k r)
    P_l(cos theta), the fields per degree l are c_l h_l(k0 r) outside (h_l = j_l + i y_l)
    and a_l j_l(k1 r) inside (total), and continuity of u and of its radial derivative at
    r = R gives the same c_l, a_l as the disk with J_n, H_n replaced by j_l, h_l."""
    k0 = omega
    k1 = omega * np.sqrt(1.0 - m0)
    if lmax is None:
        lmax = int(k1 * R + 4.0 * (k1 * R) ** (1.0 / 3.0) + 15)
    dx = [np.asarray(X1) - centre[0], np.asarray(X2) - centre[1], np.asarray(X3) - centre[2]]
    r = np.sqrt(dx[0] ** 2 + dx[1] ** 2 + dx[2] ** 2)
    rs = np.where(r > 0, r, 1.0)
    ct = np.where(r > 0, dx[0] / rs, 1.0)
    inside = r < R
    u = np.zeros(r.shape, dtype=np.complex128)
    pref = np.exp(1j * omega * centre[0])
    for l in range(lmax + 1):
        j0, j1 = sp.spherical_jn(l, k0 * R), sp.spherical_jn(l, k1 * R)
        dj0, dj1 = sp.spherical_jn(l, k0 * R, True), sp.spherical_jn(l, k1 * R, True)
        h0 = j0 + 1j * sp.spherical_yn(l, k0 * R)
        dh0 = dj0 + 1j * sp.spherical_yn(l, k0 * R, True)
        cl = (k1 * dj1 * j0 - k0 * dj0 * j1) / (k0 * dh0 * j1 - k1 * dj1 * h0)
        al = (j0 + cl * h0) / j1
        w = (2 * l + 1) * 1j ** (l % 4) * sp.eval_legendre(l, ct)
        ro, ri = r[~inside], r[inside]
        u[~inside] += pref * w[~inside] * cl * (sp.spherical_jn(l, k0 * ro) + 1j * sp.spherical_yn(l, k0 * ro))
        u[inside] += pref * w[inside] * (al * sp.spherical_jn(l, k1 * ri) - sp.spherical_jn(l, k0 * ri))
    return u
