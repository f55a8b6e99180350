"""Analytic fields the oracle is pinned against (FP64 NumPy).

TEST INFRASTRUCTURE, like the rest of ``oracle/``.

Units follow the general form of the paper's Eqs. E and B: E carries k_e
(1/(4 pi eps0), the paper's 1/(4 pi)), B carries k_b (mu0/(4 pi)); the fields
of moving charges below assume the Maxwell-consistent choice k_b = k_e / c^2.

* ``coulomb``        static point charge: E = k_e q D / R^3
* ``biot_savart``    static current element J dV: B = k_b dV J x D / R^3
* ``gauss_sphere``   spherical Gaussian charge (Gauss's law with an erf
                     enclosed charge)
* ``lienard_wiechert`` point charge in uniform motion, fields at the present
                     position (Heaviside form)
* ``gaussian_lw``    the same for a rigidly moving Gaussian blob, by
                     tensor Gauss-Hermite quadrature of the point field
* ``hertz_dipole``   oscillating point dipole p(t) z-hat with near,
                     intermediate and far terms, times the Gaussian form
                     factor exp(-(omega sigma / c)^2 / 2) of a smeared dipole
* ``uniform_box``    static field of a uniformly charged rectangular box
                     (the saturated state of the paper's step-on sources,
                     Sec. 3.1), in closed form
* ``xoy_deviation``  the paper's error norm in the XOY plane (Eq. norms)
* ``step_box``       E and B of uniform rho and J switched on at t = 0 in a
                     box (the paper's Sec. 3.1 sources) at any time, from
                     the sphere-box moments of the switch-on front
* ``jefimenko_ball``  the same for sources that switch on continuously at
                     t = 0: the integral over the part of the box inside
                     the ball R < c t, in spherical coordinates about each
                     observation point (accurate while the front crosses)
* ``jefimenko_quadrature``  the continuous Eqs. E and B over a box for
                     analytic sources, by tensor Gauss-Legendre quadrature
                     (spectrally accurate while the integrand is smooth)
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def _as_pts(obs):
    return np.asarray(obs, dtype=np.float64).reshape(-1, 3)


def coulomb(q, rs, obs, k_e=1.0):
    D = _as_pts(obs) - np.asarray(rs, dtype=np.float64)
    R = np.linalg.norm(D, axis=1)
    return k_e * q * D / R[:, None] ** 3


def biot_savart(Jvec, dV, rs, obs, k_b=1.0):
    D = _as_pts(obs) - np.asarray(rs, dtype=np.float64)
    R = np.linalg.norm(D, axis=1)
    return k_b * dV * np.cross(np.asarray(Jvec, dtype=np.float64)[None, :], D) / R[:, None] ** 3


def gauss_sphere(Q, sigma, center, obs, k_e=1.0):
    """E of a spherical Gaussian charge Q with standard deviation sigma."""
    D = _as_pts(obs) - np.asarray(center, dtype=np.float64)
    r = np.linalg.norm(D, axis=1)
    x = r / sigma
    q_enc = Q * (erf(x / math.sqrt(2.0)) - math.sqrt(2.0 / math.pi) * x * np.exp(-0.5 * x * x))
    return k_e * q_enc[:, None] * D / r[:, None] ** 3


def lienard_wiechert(q, pos_now, v, obs, c=1.0, k_e=1.0, k_b=None):
    """Fields of a point charge moving with constant velocity v, located at
    ``pos_now`` at the observation time (Heaviside's form of the
    Lienard-Wiechert field).  pos_now may be [3] or [n, 3] (per point)."""
    if k_b is None:
        k_b = k_e / (c * c)
    v = np.asarray(v, dtype=np.float64)
    P = _as_pts(obs) - np.asarray(pos_now, dtype=np.float64)
    R = np.linalg.norm(P, axis=1)
    beta2 = float(v @ v) / (c * c)
    vn = math.sqrt(float(v @ v))
    if vn > 0:
        cos_psi = (P @ v) / (R * vn)
        sin2 = 1.0 - cos_psi ** 2
    else:
        sin2 = np.zeros_like(R)
    E = k_e * q * (1.0 - beta2) * P / (R[:, None] ** 3 * (1.0 - beta2 * sin2)[:, None] ** 1.5)
    B = (k_b / k_e) * np.cross(v[None, :], E)
    return E, B


def gaussian_lw(q, sigma, center_now, v, obs, c=1.0, k_e=1.0, k_b=None, n_gh=12):
    """Fields of a Gaussian charge blob (per-axis standard deviations
    ``sigma``) moving rigidly with velocity v, centred at ``center_now`` at the
    observation time: the point field above averaged over the blob by a
    tensor Gauss-Hermite rule with n_gh nodes per axis."""
    sig = np.broadcast_to(np.asarray(sigma, dtype=np.float64), (3,))
    x, w = np.polynomial.hermite.hermgauss(n_gh)
    nodes = np.sqrt(2.0) * x
    wts = w / np.sqrt(np.pi)
    obs = _as_pts(obs)
    E = np.zeros_like(obs)
    B = np.zeros_like(obs)
    cen = np.asarray(center_now, dtype=np.float64)
    for i in range(n_gh):
        for j in range(n_gh):
            for k in range(n_gh):
                off = np.array([nodes[i] * sig[0], nodes[j] * sig[1], nodes[k] * sig[2]])
                wt = wts[i] * wts[j] * wts[k]
                e, b = lienard_wiechert(q, cen + off, v, obs, c=c, k_e=k_e, k_b=k_b)
                E += wt * e
                B += wt * b
    return E, B


def hertz_dipole(p0, omega, obs, t, c=1.0, k_e=1.0, k_b=None, sigma=0.0, phase=0.0):
    """Oscillating dipole p(t) = p0 cos(omega t + phase) z-hat at the origin.

    E = k_e [ (3(p.n)n - p)/r^3 + (3(p'.n)n - p')/(c r^2) + ((p''.n)n - p'')/(c^2 r) ]
    B = k_b [ p' x n / r^2 + p'' x n / (c r) ]
    with p, p', p'' taken at t - r/c, times exp(-(omega sigma/c)^2/2) for a
    dipole smeared by a spherical Gaussian of standard deviation sigma.
    """
    if k_b is None:
        k_b = k_e / (c * c)
    obs = _as_pts(obs)
    r = np.linalg.norm(obs, axis=1)
    n = obs / r[:, None]
    tr = t - r / c
    ph = omega * tr + phase
    p = p0 * np.cos(ph)
    pd = -p0 * omega * np.sin(ph)
    pdd = -p0 * omega * omega * np.cos(ph)
    z = np.array([0.0, 0.0, 1.0])
    nz = n[:, 2]

    def vec(a):
        return a[:, None] * z[None, :]

    E = (vec(p) * -1 + 3 * (p * nz)[:, None] * n) / r[:, None] ** 3
    E += (vec(pd) * -1 + 3 * (pd * nz)[:, None] * n) / (c * r[:, None] ** 2)
    E += (vec(pdd) * -1 + (pdd * nz)[:, None] * n) / (c * c * r[:, None])
    B = np.cross(vec(pd), n) / r[:, None] ** 2 + np.cross(vec(pdd), n) / (c * r[:, None])
    F = math.exp(-0.5 * (omega * sigma / c) ** 2)
    return k_e * F * E, k_b * F * B


def _rect_inv_r(u, va, vb, wa, wb):
    """Integral of 1/sqrt(u^2 + v^2 + w^2) over v in [va, vb], w in [wa, wb],
    from the antiderivative G = v ln(w + r) + w ln(v + r) - u atan(v w / (u r))
    (d^2 G / dv dw = 1/r; the u term vanishes with u)."""
    def G(v, w):
        r = np.sqrt(u * u + v * v + w * w)
        safe_u = np.where(u == 0.0, 1.0, u)
        at = np.where(u == 0.0, 0.0, u * np.arctan(v * w / (safe_u * r)))
        return v * np.log(w + r) + w * np.log(v + r) - at

    return G(vb, wb) - G(va, wb) - G(vb, wa) + G(va, wa)


def uniform_box(obs, lo, hi, rho=1.0, k_e=1.0):
    """E of charge density rho filling the box [lo, hi] (static Coulomb field,
    the rho/R^3 term of Eq. E integrated over the box).

    Along axis a the kernel (x_a - x'_a)/R^3 integrates in closed form to
    1/R(x_a - hi_a) - 1/R(x_a - lo_a); the remaining integral of 1/R over the
    box's face rectangle is _rect_inv_r.  Valid off the box's edge lines
    (every point strictly inside or outside works; cell centres qualify).
    A uniform current J in the same box gives B = (k_b / (k_e rho)) J x E."""
    P = _as_pts(obs)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    E = np.empty_like(P)
    for a in range(3):
        b, c = (a + 1) % 3, (a + 2) % 3
        va, vb = P[:, b] - hi[b], P[:, b] - lo[b]
        wa, wb = P[:, c] - hi[c], P[:, c] - lo[c]
        E[:, a] = _rect_inv_r(P[:, a] - hi[a], va, vb, wa, wb) - _rect_inv_r(P[:, a] - lo[a], va, vb, wa, wb)
    return k_e * rho * E


def xoy_deviation(A, A_ref):
    """The paper's comparison in the XOY plane (Eq. norms): per point
    |A_ref - A| = sqrt(dA_x^2 + dA_y^2) and |A_ref| = sqrt(A_x^2 + A_y^2), z
    components left out.  Returns (max deviation, max |A_ref|) over the
    points given; their ratio is the relative deviation the paper quotes."""
    A = np.asarray(A, dtype=np.float64).reshape(-1, 3)
    R = np.asarray(A_ref, dtype=np.float64).reshape(-1, 3)
    dev = np.hypot(R[:, 0] - A[:, 0], R[:, 1] - A[:, 1])
    nrm = np.hypot(R[:, 0], R[:, 1])
    return float(dev.max()), float(nrm.max())


def _arcs_in_rectangle(rho, ax, bx, ay, by):
    """Angles phi in [-pi, pi] (as intervals) where the circle point
    (rho cos phi, rho sin phi) lies in [ax, bx] x [ay, by]."""
    cuts = [-math.pi, math.pi]
    for cv in (ax, bx):
        if abs(cv) <= rho:
            a = math.acos(max(-1.0, min(1.0, cv / rho)))
            cuts += [a, -a]
    for cv in (ay, by):
        if abs(cv) <= rho:
            a = math.asin(max(-1.0, min(1.0, cv / rho)))
            cuts += [a, (math.pi - a) if a >= 0 else (-math.pi - a)]
    cuts = sorted(set(cuts))
    out = []
    for p0, p1 in zip(cuts[:-1], cuts[1:]):
        m = 0.5 * (p0 + p1)
        x, y = rho * math.cos(m), rho * math.sin(m)
        if p1 > p0 and ax <= x <= bx and ay <= y <= by:
            out.append((p0, p1))
    return out


def sphere_box_moments(r, R, lo, hi, n_gl=16):
    """For the sphere of radius R about r: the solid angle C of directions n
    with r - R n inside the box [lo, hi], and the vector A = integral of n
    over those directions.  On the unit sphere dOmega = du dphi with
    u = n_z; each z-slice is a circle whose part inside the box's (x, y)
    rectangle is a union of arcs in closed form, and the u integral runs
    piecewise (Gauss-Legendre) between the u where the arcs change."""
    r = np.asarray(r, dtype=np.float64)
    a = (r - np.asarray(hi, dtype=np.float64)) / R
    b = (r - np.asarray(lo, dtype=np.float64)) / R
    u0, u1 = max(a[2], -1.0), min(b[2], 1.0)
    if u0 >= u1:
        return 0.0, np.zeros(3)
    cuts = {u0, u1}
    for cv in (a[0], b[0], a[1], b[1]):
        if abs(cv) < 1.0:
            cuts |= {math.sqrt(1.0 - cv * cv), -math.sqrt(1.0 - cv * cv)}
    for cx in (a[0], b[0]):
        for cy in (a[1], b[1]):
            q = cx * cx + cy * cy
            if q < 1.0:
                cuts |= {math.sqrt(1.0 - q), -math.sqrt(1.0 - q)}
    cuts = sorted(x for x in cuts if u0 <= x <= u1)
    x, w = np.polynomial.legendre.leggauss(n_gl)
    C, A = 0.0, np.zeros(3)
    for p, q in zip(cuts[:-1], cuts[1:]):
        for xi, wi in zip(x, w):
            u = 0.5 * (p + q) + 0.5 * (q - p) * xi
            ww = 0.5 * (q - p) * wi
            rho = math.sqrt(max(0.0, 1.0 - u * u))
            for p0, p1 in _arcs_in_rectangle(rho, a[0], b[0], a[1], b[1]):
                C += ww * (p1 - p0)
                A += ww * np.array([rho * (math.sin(p1) - math.sin(p0)),
                                    rho * (math.cos(p0) - math.cos(p1)), u * (p1 - p0)])
    return C, A


def step_box(r, t, lo, hi, J0, n_gl=16, k_e=1.0, k_b=1.0):
    """E and B at point r and time t (c = 1) of rho = 1 and J = J0 switched on
    at t = 0 inside the box [lo, hi] (the paper's Sec. 3.1 sources).

    With n the unit vector from source to observer and R the distance, the
    terms of Eqs. E and B become, for step sources (d/dt = delta(t_r)),
      E = Int_0^t A(R) dR + t A(t) - J0 t C(t)
      B = J0 x ( Int_0^t A(R) dR + t A(t) )
    where C(R), A(R) are the sphere-box moments above: the Coulomb and
    Biot-Savart terms gather the ball R < t already switched on, the
    derivative terms the switch-on front R = t.  The R integral runs
    piecewise between the distances at which the sphere meets a face, an
    edge or a corner of the box."""
    r = np.asarray(r, dtype=np.float64)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    J0 = np.asarray(J0, dtype=np.float64)
    cuts = {0.0, float(t)}
    for a in range(3):
        cuts |= {abs(r[a] - lo[a]), abs(r[a] - hi[a])}
        b, c = (a + 1) % 3, (a + 2) % 3
        for fb in (lo[b], hi[b]):
            for fc in (lo[c], hi[c]):
                cuts.add(math.hypot(r[b] - fb, r[c] - fc))
    for fx in (lo[0], hi[0]):
        for fy in (lo[1], hi[1]):
            for fz in (lo[2], hi[2]):
                cuts.add(math.sqrt((r[0] - fx) ** 2 + (r[1] - fy) ** 2 + (r[2] - fz) ** 2))
    cuts = sorted(x for x in cuts if 0.0 <= x <= t)
    x, w = np.polynomial.legendre.leggauss(n_gl)
    ball = np.zeros(3)
    for p, q in zip(cuts[:-1], cuts[1:]):
        for xi, wi in zip(x, w):
            R = 0.5 * (p + q) + 0.5 * (q - p) * xi
            ball += 0.5 * (q - p) * wi * sphere_box_moments(r, R, lo, hi, n_gl)[1]
    Ct, At = sphere_box_moments(r, t, lo, hi, n_gl) if t > 0 else (0.0, np.zeros(3))
    return k_e * (ball + t * At - J0 * t * Ct), k_b * np.cross(J0, ball + t * At)


def _box_cuts(r, lo, hi):
    """Distances from r at which a sphere about r meets a face plane, an edge
    line or a corner of the box [lo, hi]."""
    cuts = set()
    for a in range(3):
        cuts |= {abs(r[a] - lo[a]), abs(r[a] - hi[a])}
        b, c = (a + 1) % 3, (a + 2) % 3
        for fb in (lo[b], hi[b]):
            for fc in (lo[c], hi[c]):
                cuts.add(math.hypot(r[b] - fb, r[c] - fc))
    for fx in (lo[0], hi[0]):
        for fy in (lo[1], hi[1]):
            for fz in (lo[2], hi[2]):
                cuts.add(math.sqrt((r[0] - fx) ** 2 + (r[1] - fy) ** 2 + (r[2] - fz) ** 2))
    return cuts


def jefimenko_ball(obs, t, lo, hi, sources, n_gl=16, c=1.0, k_e=1.0, k_b=1.0):
    """E and B of the continuous Eqs. E and B (as ``jefimenko_quadrature``)
    for sources that are zero before t = 0 and continuous in time there
    (their derivatives may jump): only the part of the box inside the ball
    R < c t contributes.  In spherical coordinates about each observation
    point, r' = r - R n with dV' = R^2 dR dOmega and dOmega = du dphi
    (u = n_z), the integrands become
      E: n rho + n drho R / c - dJ R / c^2,   B: (J + dJ R / c) x n
    and every layer is smooth: R runs piecewise between the distances at
    which the sphere meets a face, an edge or a corner of the box (and c t),
    u between the values where the slice's arcs inside the box change, phi
    over those arcs, each piece by Gauss-Legendre."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    x, w = np.polynomial.legendre.leggauss(int(n_gl))
    obs = _as_pts(obs)
    E = np.zeros_like(obs)
    B = np.zeros_like(obs)
    for k, r in enumerate(obs):
        cuts = sorted(v for v in _box_cuts(r, lo, hi) | {0.0, c * t} if 0.0 <= v <= c * t)
        for p, q in zip(cuts[:-1], cuts[1:]):
            for xi, wi in zip(x, w):
                R = 0.5 * (p + q) + 0.5 * (q - p) * xi
                wR = 0.5 * (q - p) * wi
                a = (r - hi) / R
                b = (r - lo) / R
                u0, u1 = max(a[2], -1.0), min(b[2], 1.0)
                if u0 >= u1:
                    continue
                uc = {u0, u1}
                for cv in (a[0], b[0], a[1], b[1]):
                    if abs(cv) < 1.0:
                        uc |= {math.sqrt(1.0 - cv * cv), -math.sqrt(1.0 - cv * cv)}
                for cx in (a[0], b[0]):
                    for cy in (a[1], b[1]):
                        qq = cx * cx + cy * cy
                        if qq < 1.0:
                            uc |= {math.sqrt(1.0 - qq), -math.sqrt(1.0 - qq)}
                uc = sorted(v for v in uc if u0 <= v <= u1)
                dirs, wts = [], []
                for up, uq in zip(uc[:-1], uc[1:]):
                    for xj, wj in zip(x, w):
                        u = 0.5 * (up + uq) + 0.5 * (uq - up) * xj
                        wu = 0.5 * (uq - up) * wj
                        rho_u = math.sqrt(max(0.0, 1.0 - u * u))
                        for p0, p1 in _arcs_in_rectangle(rho_u, a[0], b[0], a[1], b[1]):
                            phi = 0.5 * (p0 + p1) + 0.5 * (p1 - p0) * x
                            dirs.append(np.stack([rho_u * np.cos(phi), rho_u * np.sin(phi),
                                                  np.full_like(phi, u)], axis=1))
                            wts.append(wR * wu * 0.5 * (p1 - p0) * w)
                if not dirs:
                    continue
                n = np.concatenate(dirs)
                ww = np.concatenate(wts)
                rho, drho, J, dJ = sources(r - R * n, np.full(len(n), t - R / c))
                e = n * (rho + drho * R / c)[:, None] - dJ * (R / (c * c))
                bb = np.cross(J + dJ * (R / c), n)
                E[k] += ww @ e
                B[k] += ww @ bb
    return k_e * E, k_b * B


def jefimenko_quadrature(obs, t, lo, hi, sources, n_gl=32, c=1.0, k_e=1.0, k_b=1.0):
    """E and B of the continuous Jefimenko equations (paper Eqs. E and B, with
    t_r = t - R/c of Eq. tr) for sources filling the box [lo, hi]:

      E = k_e Int [ D rho/R^3 + D drho/(c R^2) - dJ/(c^2 R) ] dV'
      B = k_b Int [ J/R^3 + dJ/(c R^2) ] x D dV'

    D = r - r', every source quantity at (r', t_r).  sources(points, t_r)
    returns (rho, drho_dt, J, dJ_dt) with shapes [m], [m], [m, 3], [m, 3].
    The integral is a tensor Gauss-Legendre rule with n_gl nodes per axis:
    spectrally accurate for observation points outside the box and times at
    which no switch-on front (a jump of the sources in time) crosses the box.
    """
    x, w = np.polynomial.legendre.leggauss(int(n_gl))
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    half, mid = (hi - lo) / 2.0, (hi + lo) / 2.0
    ax = [mid[a] + half[a] * x for a in range(3)]
    wa = [half[a] * w for a in range(3)]
    X, Y, Z = np.meshgrid(ax[0], ax[1], ax[2], indexing="ij")
    S = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    W = (wa[0][:, None, None] * wa[1][None, :, None] * wa[2][None, None, :]).ravel()
    obs = _as_pts(obs)
    E = np.zeros_like(obs)
    B = np.zeros_like(obs)
    for k, o in enumerate(obs):
        D = o - S
        R = np.linalg.norm(D, axis=1)
        rho, drho, J, dJ = sources(S, t - R / c)
        e = D * (rho / R ** 3 + drho / (c * R ** 2))[:, None] - dJ / (c * c * R)[:, None]
        b = np.cross(J / R[:, None] ** 3 + dJ / (c * R[:, None] ** 2), D)
        E[k] = W @ e
        B[k] = W @ b
    return k_e * E, k_b * B


def rel_l2(a, b):
    """Normwise relative L2 error ||a - b|| / ||b||."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a - b))
