"""Pins of the FP64 oracle against values that the paper and the mathematics
fix independently of the oracle: published known-answer vectors, textbook
closed forms, library routines (scipy) and brute force on tiny inputs.

Every check lives in a ``check_*`` function so that the mutation tests in
``test_oracle_mutants.py`` can run the same checks against builds of the
oracle with a planted mistake.  CPU only.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, ndimage, special, stats

from oracle import oracle as orc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ----------------------------------------------------------------- helpers
def scipy_window(A, B, C, w, b):
    """W(w) of Eq. 4 for the lobe of Eq. 5 normalised over [-pi/2, pi/2],
    integrated by scipy's QUADPACK; Z through log-gamma."""
    S = 1.0 - A - B
    lo, hi = max(w - b / 2, -math.pi / 2), min(w + b / 2, math.pi / 2)
    if hi <= lo:
        return 0.0
    f = lambda a: A + B * math.cos(a) + S * max(math.cos(a), 0.0) ** C
    pts = [0.0] if lo < 0.0 < hi else None
    v, _ = integrate.quad(f, lo, hi, epsabs=1e-15, epsrel=1e-13, limit=1000, points=pts)
    Z = A * math.pi + 2 * B + S * math.sqrt(math.pi) * math.exp(special.gammaln((C + 1) / 2) - special.gammaln(C / 2 + 1))
    return v / Z


def textbook_fresnel(n1, n2, ti):
    """Unpolarised power reflectance from the angle forms of the Fresnel equations."""
    if ti == 0.0:
        return ((n1 - n2) / (n1 + n2)) ** 2
    st = n1 / n2 * math.sin(ti)
    if st >= 1.0:
        return 1.0
    tt = math.asin(st)
    rs = math.sin(ti - tt) ** 2 / math.sin(ti + tt) ** 2
    rp = math.tan(ti - tt) ** 2 / math.tan(ti + tt) ** 2
    return 0.5 * (rs + rp)


def make_material(eps_r=1.0, tan_d=0.0, A=0.6, B=0.1, C=30.0, pec=False):
    return dict(eps_r=eps_r, loss_tangent=tan_d, A=A, B=B, C=C, pec=pec)


WALL = dict(A=0.6, B=0.1, C=30.0)
METAL_LOBE = dict(A=0.0, B=0.0, C=2000.0)


def base_params(**kw):
    p = dict(n_azimuth=1, rays_per_beam=1, max_bounces=1, n_bins=2000, beam_width=math.radians(10.0),
             beam_prob=0.9, elevation=0.0, bin_size=0.01, t_min=1e-4, min_energy=0.0, freq_hz=76.5e9,
             blur_sigma_bins=0.0, az_pattern_sigma=0.0, noise_sys=0.0, noise_amb=0.0, multipath=False,
             refraction=True, speckle=False, noise=False, seed=0x5EED, scan_id=0, beam_aspect=1.0)
    p.update(kw)
    for k in ("beam_width", "beam_prob", "elevation", "bin_size", "t_min", "freq_hz", "beam_aspect"):
        p[k] = float(np.float32(p[k]))
    return p


POSE0 = dict(p=(0.0, 0.0, 0.0), q=(1.0, 0.0, 0.0, 0.0))


class Soup:
    """Tiny triangle soup for pin scenes."""

    def __init__(self):
        self.v, self.t, self.m = [], [], []

    def quad(self, centre, u, v, half, normal, mat):
        c = np.asarray(centre, float)
        u = np.asarray(u, float) * half
        v = np.asarray(v, float) * half
        P = [c - u - v, c + u - v, c + u + v, c - u + v]
        for a, b, cc in ((0, 1, 2), (0, 2, 3)):
            A, B, Cc = P[a], P[b], P[cc]
            if np.dot(np.cross(B - A, Cc - A), normal) < 0:
                B, Cc = Cc, B
            n0 = len(self.v)
            self.v += [A, B, Cc]
            self.t.append((n0, n0 + 1, n0 + 2))
            self.m.append(mat)

    def arrays(self):
        return (np.asarray(self.v, np.float32), np.asarray(self.t, np.uint32), np.asarray(self.m, np.uint16))


def frame(d):
    """Two unit vectors orthogonal to d and to each other."""
    d = np.asarray(d, float)
    a = np.array([0.0, 0.0, 1.0]) if abs(d[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
    u = np.cross(d, a)
    u /= np.linalg.norm(u)
    v = np.cross(d, u)
    return u, v


def plane_distance(soup, tri, o, d):
    """Distance along d from o to the plane of triangle tri as stored (float32)."""
    v, t, _ = soup.arrays()
    a, b, c = (v[t[tri, i]].astype(np.float64) for i in range(3))
    n = np.cross(b - a, c - a)
    return float(np.dot(a - o, n) / np.dot(d, n))


def single_return(img):
    nz = np.nonzero(img)[0]
    return nz, img[nz]


# ----------------------------------------------------------------- Philox
def check_philox_kat():
    for row in _golden_rows("philox4x32_10_kat.txt"):
        vals = [int(x, 16) for x in row]
        out = orc.philox(vals[0:4], vals[4:6])
        assert [int(x) for x in out] == vals[6:10], (row, [hex(int(x)) for x in out])


def check_u24():
    assert orc.u24(0) == 2.0 ** -24
    assert orc.u24(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    rng = np.random.default_rng(1)
    for x in rng.integers(0, 2 ** 32, size=200, dtype=np.uint64):
        u = orc.u24(int(x))
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u               # exact in float32 as well
        assert (u * 2 ** 24 - 1) / 2 == (int(x) >> 9)   # uses the top 23 bits


# ----------------------------------------------------------------- D3 (Eq. 2)
def check_d3_sigma():
    # sqrt(2) erfinv(P) is the (1+P)/2 quantile of N(0,1)
    q = stats.norm.ppf(0.95)
    assert abs(math.sqrt(2) * orc.erfinv(0.9) - q) < 1e-12
    assert abs(orc.d3_sigma(math.radians(10), 0.9) - math.radians(5) / q) < 1e-15
    assert abs(math.degrees(orc.d3_sigma(math.radians(10), 0.9)) - 3.0397841595588) < 1e-9
    assert orc.d3_sigma(0.0, 0.9) == 0.0


def check_d3_statistics(n=40000):
    p = base_params(n_azimuth=1, rays_per_beam=n)
    sigma = orc.d3_sigma(p["beam_width"], p["beam_prob"])
    r = np.empty(n)
    w = np.empty(n)
    ang = np.empty(n)
    axis = orc.beam_axis(p, POSE0, 0)
    for k in range(n):
        o, d, r[k], w[k] = orc.d3_ray(p, POSE0, 0, k)
        ang[k] = math.atan2(np.linalg.norm(np.cross(d, axis)), np.dot(d, axis))
    assert np.allclose(axis, [1, 0, 0])
    z = r / sigma
    # E[r^2] = sigma^2 (4 standard errors)
    assert abs(np.mean(z ** 2) - 1.0) < 4 * math.sqrt(2.0 / n)
    # P(|r| <= b/2) = P
    frac = np.mean(np.abs(r) <= p["beam_width"] / 2)
    assert abs(frac - 0.9) < 4 * math.sqrt(0.09 / n)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    assert stats.kstest((w + math.pi) / (2 * math.pi), "uniform").pvalue > 1e-4
    # the ray's angle to the beam axis is |r| to second order
    assert np.max(np.abs(ang - np.abs(r))) < 0.01 * np.max(np.abs(r)) ** 2 + 1e-12
    # each component carries half the variance: r cos w and r sin w
    assert abs(np.mean((r * np.cos(w)) ** 2) / sigma ** 2 - 0.5) < 4 * math.sqrt(0.5 / n)


def check_d3_pose_and_azimuth():
    p = base_params(n_azimuth=8, elevation=math.radians(5.0), beam_width=0.0)
    yaw = 0.3
    pz = dict(p=(1.0, 2.0, 3.0), q=(math.cos(yaw / 2), 0.0, 0.0, math.sin(yaw / 2)))
    for a in range(8):
        o, d, r, _ = orc.d3_ray(p, pz, a, 0)
        phi = 2 * math.pi * a / 8 + yaw
        el = float(np.float32(math.radians(5.0)))
        expect = [math.cos(el) * math.cos(phi), math.cos(el) * math.sin(phi), math.sin(el)]
        assert r == 0.0
        assert np.allclose(o, [1, 2, 3])
        assert np.allclose(d, expect, atol=1e-14)


# ----------------------------------------------------------------- Fresnel / Snell
def check_fresnel_closed_forms():
    for name, n1, n2, deg, R in _golden_rows("fresnel_brdf_pins.txt")[:4]:
        n1, n2, ti, R = float(n1), float(n2), math.radians(float(deg)), float(R)
        got, ct, tir = orc.fresnel(n1, n2, math.cos(ti))
        assert not tir
        assert abs(got - R) < 1e-12, name
        assert abs(got - textbook_fresnel(n1, n2, ti)) < 1e-12, name
    # Brewster: the p reflectance vanishes, R = Rs / 2
    R, _, _ = orc.fresnel(1.0, 2.0, math.cos(math.atan(2.0)))
    assert abs(R - 0.18) < 1e-12
    # critical angle inside n = 2: 30 deg
    assert orc.fresnel(2.0, 1.0, math.cos(math.radians(30.0) + 1e-9))[2]
    assert not orc.fresnel(2.0, 1.0, math.cos(math.radians(30.0) - 1e-9))[2]
    assert orc.fresnel(2.0, 1.0, math.cos(math.radians(45.0)))[0] == 1.0
    # reciprocity: the same interface seen from both sides reflects the same
    for deg in (5, 17, 29):
        ti = math.radians(deg)
        R12, ct, _ = orc.fresnel(2.0, 1.0, math.cos(ti))
        R21, _, _ = orc.fresnel(1.0, 2.0, ct)
        assert abs(R12 - R21) < 1e-12
    # equal indices: no interface
    assert orc.fresnel(1.5, 1.5, 0.3)[0] < 1e-30


def check_snell():
    rng = np.random.default_rng(7)
    for _ in range(200):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        if np.dot(d, n) > 0:
            d = -d
        cos_i = -np.dot(d, n)
        n1, n2 = rng.uniform(1, 3, size=2)
        R, cos_t, tir = orc.fresnel(n1, n2, cos_i)
        refl = orc.reflect(d, n)
        assert abs(np.linalg.norm(refl) - 1) < 1e-12
        assert abs(np.dot(refl, n) - cos_i) < 1e-12                 # theta1 = theta0
        assert abs(np.dot(np.cross(d, n), refl)) < 1e-12           # plane of incidence
        if tir:
            assert (n1 / n2) * math.sqrt(max(0.0, 1 - cos_i ** 2)) >= 1 - 1e-12
            continue
        t = orc.refract(d, n, n1 / n2, cos_i, cos_t)
        assert abs(np.linalg.norm(t) - 1) < 1e-12
        sin_i = np.linalg.norm(np.cross(d, n))
        sin_t = np.linalg.norm(np.cross(t, n))
        assert abs(n1 * sin_i - n2 * sin_t) < 1e-12                # Snell
        assert np.dot(t, n) < 0                                    # goes through
        assert abs(np.dot(np.cross(d, n), t)) < 1e-12              # plane of incidence


# ----------------------------------------------------------------- BRDF (Eq. 3-5)
def check_brdf_normalisation():
    for A, B, C in ((0.6, 0.1, 30.0), (0.6, 0.1, 70.0), (0.01, 0.95, 1900.0), (0.0, 0.0, 2000.0),
                    (0.2, 0.3, 2.5), (1.0, 0.0, 0.0), (0.0, 1.0, 5.0)):
        m = make_material(A=A, B=B, C=C)
        v, _ = integrate.quad(lambda w: orc.brdf_density(m, w), -math.pi / 2, math.pi / 2, points=[0.0],
                              limit=2000, epsabs=1e-13, epsrel=1e-12)
        assert abs(v - 1.0) < 1e-9, (A, B, C, v)
        assert abs(orc.brdf_window(m, 0.0, math.pi) - 1.0) < 1e-10
    # Wallis: integral of cos^n over [-pi/2, pi/2]
    for nn in range(0, 12):
        dfac = lambda k: 1 if k <= 0 else k * dfac(k - 2)
        exact = (math.pi if nn % 2 == 0 else 2.0) * dfac(nn - 1) / dfac(nn)
        assert abs(orc.int_cospow(nn, -math.pi / 2, math.pi / 2) - exact) < 1e-12


def check_brdf_window_pins():
    rows = _golden_rows("fresnel_brdf_pins.txt")[4:]
    b10 = math.radians(10.0)
    bt = math.radians(2.960736528512652)
    for name, A, B, C, w10, wt in rows:
        m = make_material(A=float(A), B=float(B), C=float(C))
        assert abs(orc.brdf_window(m, 0.0, b10) - float(w10)) < 1e-12, name
        assert abs(orc.brdf_window(m, 0.0, bt) - float(wt)) < 1e-12, name
    m = make_material(**WALL)
    for w in (-1.2, -0.3, 0.2, 0.7, 1.5):
        assert abs(orc.brdf_window(m, w, b10) - scipy_window(0.6, 0.1, 30.0, w, b10)) < 1e-12
        assert abs(orc.brdf_window(m, w, b10) - orc.brdf_window(m, -w, b10)) < 1e-14
    assert orc.brdf_window(m, math.pi / 2 + b10 / 2 + 1e-9, b10) == 0.0
    assert orc.brdf_window(m, math.pi / 2 + b10 / 2 - 1e-3, b10) > 0.0


# ----------------------------------------------------------------- intersection
def check_closest_brute_force():
    """Oracle closest hit vs a different algorithm: plane solve with numpy."""
    from paper_2310_03505_gb300 import scenes
    sc = scenes.tiny_room()
    V = sc.vertices.astype(np.float64)
    T = sc.triangles
    v0, v1, v2 = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    rng = np.random.default_rng(3)
    for _ in range(150):
        o = rng.uniform([-4.5, -4.5, 0.2], [4.5, 4.5, 2.8])
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        # solve o + t d = v0 + b1 (v1 - v0) + b2 (v2 - v0) for every triangle
        M = np.stack([-np.broadcast_to(d, v0.shape), v1 - v0, v2 - v0], axis=2)
        ok = np.abs(np.linalg.det(M)) > 1e-14
        sol = np.full((len(T), 3), np.nan)
        sol[ok] = np.linalg.solve(M[ok], (o - v0)[ok][..., None])[..., 0]
        t, b1, b2 = sol[:, 0], sol[:, 1], sol[:, 2]
        valid = ok & (t > 1e-4) & (b1 >= 0) & (b2 >= 0) & (b1 + b2 <= 1)
        tri, tt, fl = orc.closest(sc.vertices, sc.triangles, o, d)
        if not valid.any():
            assert tri is None
            continue
        tmin = np.min(t[valid])
        cand = np.nonzero(valid & (t <= tmin * (1 + 1e-12)))[0]
        assert abs(tt - tmin) < 1e-9 * max(1.0, tmin)
        if fl == 0:
            assert tri == cand.min()
        assert fl != 0 or len(cand) == 1


# ----------------------------------------------------------------- scans on pin scenes
def _scan(soup, mats, p, pose=POSE0, **kw):
    v, t, m = soup.arrays()
    return orc.scan(v, t, m, mats, pose, p, **kw)


def check_normal_incidence_plane():
    """Plane perpendicular to the drawn ray at distance D: one return at bin
    floor(D / bin) with energy R W(0): W(0) for a perfect conductor, W(0)/9
    for eps_r = 4."""
    p = base_params()
    _, d, _, _ = orc.d3_ray(p, POSE0, 0, 0)
    u, v = frame(d)
    D = 10.013
    b = p["beam_width"]                     # the float32 value both sides read
    for mat, expect in ((make_material(pec=True, **METAL_LOBE), scipy_window(0, 0, 2000, 0.0, b)),
                        (make_material(eps_r=4.0, tan_d=0.01, **WALL), scipy_window(0.6, 0.1, 30, 0.0, b) / 9.0)):
        s = Soup()
        s.quad(D * d, u, v, 2.0, -d, 0)
        r = _scan(s, [mat], p)
        nz, e = single_return(r["image"][0])
        assert list(nz) == [int(D / p["bin_size"])]
        assert abs(e[0] - expect) < 1e-9 * expect
        assert abs(r["tallies"][0, 0].sum() - 1.0) < 1e-12


def check_oblique_plane():
    """Plane tilted by theta0 = 20 deg: return R(20 deg) W(40 deg) at the range
    along the ray (traveled path: omega = theta0 + theta1)."""
    p = base_params()
    _, d, _, _ = orc.d3_ray(p, POSE0, 0, 0)
    u, v = frame(d)
    th = math.radians(20.0)
    n = -(math.cos(th) * d + math.sin(th) * u)
    D = 7.0153
    s = Soup()
    nu = np.cross(n, v)
    nu /= np.linalg.norm(nu)
    s.quad(D * d, nu, v, 3.0, n, 0)
    r = _scan(s, [make_material(eps_r=4.0, **WALL)], p)
    nz, e = single_return(r["image"][0])
    assert list(nz) == [int(D / p["bin_size"])]
    expect = textbook_fresnel(1.0, 2.0, th) * scipy_window(0.6, 0.1, 30.0, 2 * th, p["beam_width"])
    assert abs(e[0] - expect) < 1e-6 * expect


def check_slab():
    """eps_r = 4 slab of thickness t backed by a perfect conductor, normal
    incidence, multipath off: returns at D (W(0)/9), at D + 2t (optical path;
    (8/9) e^{-2 alpha t} W_metal(0)) and the internal multiple at D + 4t."""
    p = base_params(max_bounces=3)
    _, d, _, _ = orc.d3_ray(p, POSE0, 0, 0)
    u, v = frame(d)
    D, th = 5.0134, 0.0512
    s = Soup()
    s.quad(D * d, u, v, 2.0, -d, 0)                 # front face, dielectric
    s.quad((D + th) * d, u, v, 2.0, -d, 1)          # back face, metal (faces the slab)
    mats = [make_material(eps_r=4.0, tan_d=0.01, **WALL), make_material(pec=True, **METAL_LOBE)]
    r = _scan(s, mats, p)
    alpha = math.pi * 2.0 * 0.01 * p["freq_hz"] / 299792458.0
    assert abs(alpha - 16.0336) < 1e-3                       # 1/e power depth 3.12 cm
    t_front = plane_distance(s, 0, np.zeros(3), d)
    att = math.exp(-2 * alpha * (plane_distance(s, 2, np.zeros(3), d) - t_front))
    w_wall, w_metal = scipy_window(0.6, 0.1, 30, 0.0, p["beam_width"]), scipy_window(0, 0, 2000, 0.0, p["beam_width"])
    e0 = w_wall / 9
    e1 = 8 / 9 * att * w_metal
    e2 = 8 / 9 * att * (1 - w_metal) * att * (1 / 9) * w_wall
    img = r["image"][0]
    bins = [int(D / 0.01), int((D + 2 * th) / 0.01), int((D + 4 * th) / 0.01)]
    nz = np.nonzero(img)[0]
    assert list(nz) == bins, (nz, bins)
    # the third return carries 1 - W_metal(0) ~ 1e-4: quadrature error is amplified there
    for b, e, tol in zip(bins, (e0, e1, e2), (1e-9, 1e-9, 1e-7)):
        assert abs(img[b] - e) < tol * e, (b, img[b], e)
    assert abs(r["tallies"][0, 0].sum() - 1.0) < 1e-12


def check_slab_multipath():
    """Same slab with multipath on: the exit hit at bounce 2 adds an air-path
    return at ((D + 4t) + D) / 2 = D + 2t carrying T W(0) g_rx."""
    p = base_params(max_bounces=3, multipath=True)
    _, d, _, _ = orc.d3_ray(p, POSE0, 0, 0)
    u, v = frame(d)
    D, th = 5.0134, 0.0512
    s = Soup()
    s.quad(D * d, u, v, 2.0, -d, 0)
    s.quad((D + th) * d, u, v, 2.0, -d, 1)
    mats = [make_material(eps_r=4.0, tan_d=0.01, **WALL), make_material(pec=True, **METAL_LOBE)]
    r = _scan(s, mats, p)
    alpha = math.pi * 2.0 * 0.01 * p["freq_hz"] / 299792458.0
    att = math.exp(-2 * alpha * (plane_distance(s, 2, np.zeros(3), d) - plane_distance(s, 0, np.zeros(3), d)))
    w_wall, w_metal = scipy_window(0.6, 0.1, 30, 0.0, p["beam_width"]), scipy_window(0, 0, 2000, 0.0, p["beam_width"])
    sigma = p["beam_width"] / 2 / stats.norm.ppf(0.95)
    delta = math.acos(np.clip(d[0], -1, 1))                  # beam axis is +x
    g = math.exp(-0.5 * (delta / sigma) ** 2)
    e_in2 = 8 / 9 * att * (1 - w_metal) * att
    e_air = e_in2 * (8 / 9) * w_wall * g
    e1 = 8 / 9 * att * w_metal
    b = int((D + 2 * th) / 0.01)
    assert abs(r["image"][0][b] - (e1 + e_air)) < 1e-9 * (e1 + e_air)


def check_corner_reflector():
    """Perfect-conductor trihedral facing the sensor: the ray returns after
    three bounces; the third-bounce air-path return lands at half the exact
    round trip (path to the third hit + distance back) with energy
    W_metal(omega_a) g_rx, omega_a the angle between the reflected direction
    and the direction to the sensor."""
    p = base_params(max_bounces=3, multipath=True, beam_width=math.radians(1.0), bin_size=0.005)
    _, d, _, _ = orc.d3_ray(p, POSE0, 0, 0)
    # local frame: faces on x=0, y=0, z=0, normals +x, +y, +z, diagonal (1,1,1)/sqrt(3) -> -x world
    diag = np.ones(3) / math.sqrt(3)
    e1 = np.array([1.0, -1.0, 0.0]) / math.sqrt(2)
    e2 = np.cross(diag, e1)
    Rm = np.stack([-np.array([1.0, 0, 0]), np.array([0, 1.0, 0]), np.array([0, 0, 1.0])], 1) @ \
        np.stack([diag, e1, e2], 0)
    apex = np.array([8.0, 0.0, 0.0])
    s = Soup()
    planes = []
    for ax in range(3):
        nl = np.eye(3)[ax]
        ua, va = np.eye(3)[(ax + 1) % 3], np.eye(3)[(ax + 2) % 3]
        c = apex + Rm @ (0.5 * ua + 0.5 * va)
        s.quad(c, Rm @ ua, Rm @ va, 0.5, Rm @ nl, 0)
        planes.append((Rm @ nl, apex))
    mats = [make_material(pec=True, **METAL_LOBE)]
    r = _scan(s, mats, p)
    # reference path with numpy over the six stored (float32) triangles:
    # solve o + t d = a + b1 (b - a) + b2 (c - a), keep the nearest, mirror
    vs, ts, _ = s.arrays()
    tri = [tuple(vs[ts[j, i]].astype(np.float64) for i in range(3)) for j in range(len(ts))]
    o = np.zeros(3)
    dd = d.copy()
    L = 0.0
    pts = []
    skip = None
    for _ in range(3):
        best = None
        for j, (a, b_, c) in enumerate(tri):
            if j == skip:
                continue
            M = np.stack([-dd, b_ - a, c - a], 1)
            t, b1, b2 = np.linalg.solve(M, o - a)
            if t > 1e-4 and b1 >= 0 and b2 >= 0 and b1 + b2 <= 1 and (best is None or t < best[0]):
                best = (t, j)
        t, j = best
        a, b_, c = tri[j]
        n = np.cross(b_ - a, c - a)
        n /= np.linalg.norm(n)
        o = o + t * dd
        L += t
        pts.append(o)
        dd = dd - 2 * np.dot(dd, n) * n
        skip = j
    # after three mirror reflections the ray is reversed
    assert np.allclose(dd, -d, atol=1e-6)
    p3 = pts[-1]
    to_s = -p3
    dist = np.linalg.norm(to_s)
    w_a = math.atan2(np.linalg.norm(np.cross(dd, to_s)), np.dot(dd, to_s))
    sigma = p["beam_width"] / 2 / stats.norm.ppf(0.95)
    delta = math.atan2(np.linalg.norm(np.cross(p3, [1, 0, 0])), p3[0])
    g = math.exp(-0.5 * (delta / sigma) ** 2)
    expect = min(scipy_window(0.0, 0.0, 2000.0, w_a, p["beam_width"]) * g, 1.0)
    b = int((L + dist) / 2 / p["bin_size"])
    img = r["image"][0]
    assert abs(img[b] - expect) < 1e-7 * expect + 1e-12, (img[b], expect)
    assert abs((L + dist) / 2 - 8.0) < 0.05          # plane-wave picture: range of the apex
    assert abs(r["tallies"][0, 0].sum() - 1.0) < 1e-12


def check_lidar_like():
    """One bounce, one ray per azimuth, b -> narrow: the image holds a single
    return per azimuth at the plain ray-cast distance (Sec. IV-A baseline)."""
    from paper_2310_03505_gb300 import scenes
    sc = scenes.tiny_room()
    p = base_params(n_azimuth=64, rays_per_beam=1, max_bounces=1, n_bins=1142, bin_size=0.0438,
                    beam_width=math.radians(2.96), multipath=True)
    pz = dict(p=(0.0, 0.0, 0.5), q=(1.0, 0.0, 0.0, 0.0))
    r = orc.scan(sc.vertices, sc.triangles, sc.material_ids, sc.materials, pz, p)
    V = sc.vertices.astype(np.float64)
    T = sc.triangles
    v0, v1, v2 = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    nrm = np.cross(v1 - v0, v2 - v0)
    nrm /= np.linalg.norm(nrm, axis=1)[:, None]
    for a in range(64):
        o, d, _, _ = orc.d3_ray(p, pz, a, 0)
        M = np.stack([-np.broadcast_to(d, v0.shape), v1 - v0, v2 - v0], axis=2)
        sol = np.linalg.solve(M, (o - v0)[..., None])[..., 0]
        t, b1, b2 = sol.T
        valid = (t > 1e-4) & (b1 >= 0) & (b2 >= 0) & (b1 + b2 <= 1)
        j = np.nonzero(valid)[0][np.argmin(t[valid])]
        nz = np.nonzero(r["image"][a])[0]
        assert len(nz) <= 1
        th = math.acos(abs(np.dot(d, nrm[j])))
        mat = sc.materials[sc.material_ids[j]]
        R = 1.0 if mat["pec"] else textbook_fresnel(1.0, math.sqrt(mat["eps_r"]), th)
        e = R * scipy_window(mat["A"], mat["B"], mat["C"], 2 * th, p["beam_width"])
        if e > 0:
            assert list(nz) == [int(t[j] / p["bin_size"])], a
            assert abs(r["image"][a][nz[0]] - e) < 1e-7 * e + 1e-15
        else:
            assert len(nz) == 0


def check_conservation_tiny():
    from paper_2310_03505_gb300 import scenes
    sc, pz, s = scenes.config_tiny()
    r = orc.scan(sc.vertices, sc.triangles, sc.material_ids, sc.materials, pz, s, az_list=range(0, 400, 25))
    assert np.max(np.abs(r["tallies"].sum(-1) - 1.0 / s["rays_per_beam"])) < 1e-12
    assert np.all(r["tallies"] >= -1e-18)
    # every returned joule that lands in the image is in the raw image
    assert r["raw"].sum() <= r["tallies"][..., 0].sum() + 1e-12


def check_post_pass():
    """Blur / beam pattern against scipy's Gaussian filter (zero padding along
    range, wrap-around along azimuth, same truncation for sigma = 1, 2) and
    noise bounds."""
    rng = np.random.default_rng(5)
    img = rng.uniform(size=(16, 50)) * (rng.uniform(size=(16, 50)) < 0.2)
    for sig in (1.0, 2.0):
        p = base_params(n_azimuth=16, n_bins=50, blur_sigma_bins=sig)
        got = orc.post(img, p)
        ref = ndimage.gaussian_filter1d(img, sig, axis=1, mode="constant", cval=0.0, truncate=3.0)
        assert np.max(np.abs(got - ref)) < 1e-14
        p = base_params(n_azimuth=16, n_bins=50, az_pattern_sigma=sig)
        got = orc.post(img, p)
        ref = ndimage.gaussian_filter1d(img, sig, axis=0, mode="wrap", truncate=3.0)
        assert np.max(np.abs(got - ref)) < 1e-14
    p = base_params(n_azimuth=32, n_bins=100, noise=True, noise_sys=0.3, noise_amb=0.1)
    z = orc.post(np.zeros((32, 100)), p)
    assert np.all(z > 0) and np.all(z < 0.4)
    assert abs(z.mean() - 0.2) < 0.01
    # independent uniforms for the two terms: variance (0.3^2 + 0.1^2) / 12
    assert abs(z.var() - 0.1 / 12) < 0.0015


def check_db_map():
    img = np.array([1.0, 10 ** -4.0, 10 ** -2.0, 0.0, 10 ** -9.0, 2.0])
    out = orc.db_u8(img, 40.0)
    assert list(out) == [255, 0, 128, 0, 0, 255]


def check_elliptic_beam():
    """Elliptic beams (Sec. III-A, the cone stretched along an axis): with
    aspect a the inclination offsets of the D3 rays spread a times wider than
    the azimuth offsets, and the receive weight falls off as
    exp(-delta^2 / 2 sigma^2) along azimuth, exp(-delta^2 / 2 (a sigma)^2)
    along elevation; a = 1 is the circular cone."""
    n = 20000
    for aspect in (1.0, 2.0):
        p = base_params(n_azimuth=1, rays_per_beam=n, beam_aspect=aspect)
        daz = np.empty(n)
        dinc = np.empty(n)
        for k in range(n):
            _, d, _, _ = orc.d3_ray(p, POSE0, 0, k)
            daz[k] = math.atan2(d[1], d[0])
            dinc[k] = math.asin(max(-1.0, min(1.0, d[2])))
        ratio = np.var(dinc) / np.var(daz)
        assert abs(ratio / aspect ** 2 - 1.0) < 0.08, (aspect, ratio)
        sigma = orc.d3_sigma(p["beam_width"], p["beam_prob"])
        for delta in (0.5 * sigma, sigma, 2.0 * sigma):
            g_az = orc.receive_weight(p, POSE0, 0, [10 * math.cos(delta), 10 * math.sin(delta), 0.0])
            g_el = orc.receive_weight(p, POSE0, 0, [10 * math.cos(delta), 0.0, 10 * math.sin(delta)])
            assert abs(g_az - math.exp(-0.5 * (delta / sigma) ** 2)) < 1e-12
            assert abs(g_el - math.exp(-0.5 * (delta / (aspect * sigma)) ** 2)) < 1e-12
        assert abs(orc.receive_weight(p, POSE0, 0, [5.0, 0.0, 0.0]) - 1.0) < 1e-15


def _perlin_gradient(p, I, J, purpose):
    """Lattice gradient of the reading: unit vector at angle 2 pi u, u the
    uniform of Philox counter (scan_id, I, J, purpose) (generator pinned by
    the known-answer vectors)."""
    key = (p["seed"] & 0xFFFFFFFF, p["seed"] >> 32)
    x = orc.philox((p["scan_id"], I, J, purpose), key)
    th = 2.0 * math.pi * orc.u24(x[0])
    return math.cos(th), math.sin(th)


def check_perlin():
    """Perlin noise (Sec. III-C) has value 1/2 at the lattice points, slope
    there equal to the lattice gradient (from both sides), a second derivative
    that is continuous across cell borders (the quintic fade), continuity
    across the 360 degree seam, and values in [0, 1]."""
    cell = 1024
    p = base_params(n_azimuth=8 * cell, n_bins=4 * cell, noise=True, perlin=True, noise_cell_az=cell,
                    noise_cell_bins=cell, seed=0x1234ABCD5678, scan_id=3)
    v = lambda a, b, pu=4: orc.perlin(p, a % (8 * cell), b, pu)
    h = 1.0 / cell
    for pu in (4, 5):
        for I, J in ((1, 1), (5, 2), (0, 1)):
            A, B = I * cell, J * cell
            assert abs(v(A, B, pu) - 0.5) < 1e-15
            gx, gy = _perlin_gradient(p, I, J, pu)
            right = (v(A + 1, B, pu) - v(A, B, pu)) / h
            left = (v(A, B, pu) - v(A - 1, B, pu)) / h   # I = 0: across the seam
            up = (v(A, B + 1, pu) - v(A, B, pu)) / h
            down = (v(A, B, pu) - v(A, B - 1, pu)) / h
            for d_, g_ in ((right, gx), (left, gx), (up, gy), (down, gy)):
                assert abs(d_ - g_ / math.sqrt(2.0)) < 5e-3, (pu, I, J, d_, g_)
            # second derivative on both sides of the lattice line x = I (off the line y = J)
            Bq = B + cell // 3
            d2l = (v(A - 2, Bq, pu) - 2 * v(A - 1, Bq, pu) + v(A, Bq, pu)) / h ** 2
            d2r = (v(A, Bq, pu) - 2 * v(A + 1, Bq, pu) + v(A + 2, Bq, pu)) / h ** 2
            assert abs(d2l - d2r) < 0.5, (pu, I, J, d2l, d2r)
    vals = [orc.perlin(p, a, b, 4) for a in range(0, 8 * cell, 97) for b in range(0, 4 * cell, 89)]
    assert 0.0 <= min(vals) and max(vals) <= 1.0 and np.std(vals) > 0.05


def check_cook_torrance_lobe():
    """Cook-Torrance lobe (the paper's microfacet user BRDF, Sec. IV): the
    Beckmann normalisation against scipy's quadrature; unit integral; a
    purely diffuse lobe gives (sin hi - sin lo) / 2; for small roughness m
    the microfacet part tends to a Gaussian in w of variance 2 m^2, so
    W(0, b) -> erf(b / (4 m))."""
    for m in (0.1, 0.3, 0.5, 1.0):
        ref = 2.0 * integrate.quad(lambda t: orc.beckmann(t, m), -math.pi / 4, math.pi / 4, epsabs=1e-13,
                                   epsrel=1e-12, limit=400)[0]
        assert abs(orc.beckmann_norm(m) / ref - 1.0) < 1e-9, m
    for kd, m in ((0.2, 0.5), (0.0, 0.1), (1.0, 0.3)):
        mat = make_material(A=kd, B=m, C=0.0)
        mat["lobe"] = "cook_torrance"
        assert abs(orc.brdf_window(mat, 0.0, math.pi) - 1.0) < 1e-9
        assert abs(orc.brdf_window(mat, 0.3, 0.2) - orc.brdf_window(mat, -0.3, 0.2)) < 1e-12
    mat = make_material(A=1.0, B=0.3, C=0.0)
    mat["lobe"] = "cook_torrance"
    for w, b in ((0.0, 0.3), (0.7, 0.5), (-1.4, 0.6)):
        lo, hi = max(w - b / 2, -math.pi / 2), min(w + b / 2, math.pi / 2)
        assert abs(orc.brdf_window(mat, w, b) - 0.5 * (math.sin(hi) - math.sin(lo))) < 1e-12
    m = 0.01
    mat = make_material(A=0.0, B=m, C=0.0)
    mat["lobe"] = "cook_torrance"
    for b in (0.01745, 0.03, 0.06):
        assert abs(orc.brdf_window(mat, 0.0, b) - math.erf(b / (4 * m))) < 2e-3, b


def check_tabulated_lobe():
    """Tabulated lobe (Sec. III-A, a user-defined BRDF per material): a
    quadratic density is reproduced exactly (closed-form windows, also across
    w = 0), and the Eq. 5 wall lobe tabulated gives the Eq. 5 windows."""
    x = np.arange(orc.LOBE_SAMPLES) * (0.5 * math.pi / (orc.LOBE_SAMPLES - 1))
    mat = make_material()
    mat.update(lobe="table", lobe_table=1.0 + x * x)
    P = lambda u: u + u ** 3 / 3.0                      # integral of 1 + x^2 from 0
    Z = 2.0 * P(math.pi / 2)
    for w, b in ((0.0, 0.4), (0.5, 0.3), (-0.9, 0.2), (1.4, 0.5), (-0.05, 0.2)):
        lo, hi = max(w - b / 2, -math.pi / 2), min(w + b / 2, math.pi / 2)
        exact = (P(hi) - P(lo)) / Z if lo >= 0 or hi <= 0 else (P(hi) + P(-lo)) / Z
        if hi <= 0:
            exact = (P(-lo) - P(-hi)) / Z
        assert abs(orc.brdf_window(mat, w, b) - exact) < 1e-12, (w, b)
    A, B, Cc = WALL["A"], WALL["B"], WALL["C"]
    tab = make_material()
    tab.update(lobe="table", lobe_table=A + B * np.cos(x) + (1 - A - B) * np.cos(x) ** Cc)
    eq5 = make_material(**WALL)
    for w in (0.0, 0.1, 0.5, -1.0):
        for b in (0.05, math.radians(10.0)):
            assert abs(orc.brdf_window(tab, w, b) - orc.brdf_window(eq5, w, b)) < 1e-7, (w, b)


# ----------------------------------------------------------------- speckle
def _speckle_direct(p, a, k, path, bounce, word):
    """The speckle factor from its definition: -ln u of word `word` of the
    Philox4x32-10 block (pinned by the known-answer vectors) of counter
    (scan_id, a, k, 1 | (path << 8 | bounce) << 8), key (seed_lo, seed_hi)."""
    seed = int(p["seed"])
    x = orc.philox([int(p["scan_id"]), a, k, 1 | (((path << 8) | bounce) << 8)],
                   [seed & 0xFFFFFFFF, seed >> 32])
    return -math.log(orc.u24(int(x[word])))


def check_speckle_statistics():
    """Sec. III-C speckle: the factor is Exp(1) (fully developed speckle has
    an exponential intensity; mean one keeps the expected image): mean and
    variance within 4 standard errors of 1 over 100,000 factors of distinct
    counters, and a Kolmogorov-Smirnov test against Exp(1).  The two words
    of one segment's block are independent draws (correlation ~ 0)."""
    import ctypes as C
    p = base_params(speckle=True, seed=0x1234ABCD9876, scan_id=3)
    pr = orc.make_params(p)
    L = orc.lib()
    f0 = np.array([L.orc_speckle_factor(C.byref(pr), a, k, 5, 2, 0) for a in range(250) for k in range(200)])
    f1 = np.array([L.orc_speckle_factor(C.byref(pr), a, k, 5, 2, 1) for a in range(250) for k in range(200)])
    f = np.concatenate([f0, f1])
    n = f.size
    assert abs(f.mean() - 1.0) < 4.0 / math.sqrt(n), f.mean()
    # Var of the sample variance of Exp(1): (mu4 - sigma^4) / n = 8 / n
    assert abs(f.var() - 1.0) < 4.0 * math.sqrt(8.0 / n), f.var()
    assert stats.kstest(f, "expon").pvalue > 1e-3
    assert abs(np.corrcoef(f0, f1)[0, 1]) < 4.0 / math.sqrt(f0.size)
    # the counter of the definition, for both words and several segments
    for (a, k, path, bounce) in ((0, 0, 0, 0), (17, 3, 2, 1), (399, 199, 0b1011, 4), (65534, 65534, 0x7FFF, 15)):
        for w in (0, 1):
            got = L.orc_speckle_factor(C.byref(pr), a, k, path, bounce, w)
            assert got == _speckle_direct(p, a, k, path, bounce, w), (a, k, path, bounce, w)


def check_speckle_in_the_scan():
    """Speckle at the scan level.  (1) A normal-incidence metal plane, one
    ray: the speckled return is the plain return times the factor of
    segment (0, 0, path 0, bounce 0), word 0.  (2) The eps_r = 4 slab on
    metal with multipath: every return is its segment's return times that
    segment's factor, word 0 for the traveled path and word 1 for the air
    path (the air-path return of the exit hit, bounce 2, shares its bin with
    the metal's traveled-path return).  (3) Averaged over many seeds, the
    speckled return of the plane equals the plain one."""
    p = base_params(seed=0xC0FFEE, scan_id=11)
    _, d, _, _ = orc.d3_ray(p, POSE0, 0, 0)
    u, v = frame(d)
    D = 10.013
    s = Soup()
    s.quad(D * d, u, v, 2.0, -d, 0)
    mats = [make_material(pec=True, **METAL_LOBE)]
    plain = _scan(s, mats, p)["image"][0]
    b = int(D / p["bin_size"])
    spk = _scan(s, mats, {**p, "speckle": True})["image"][0]
    assert list(np.nonzero(spk)[0]) == [b]
    f = _speckle_direct(p, 0, 0, 0, 0, 0)
    assert abs(spk[b] - plain[b] * f) <= 1e-12 * plain[b] * f
    # (2) the slab with multipath
    p2 = base_params(max_bounces=3, multipath=True, seed=0x5EED77, scan_id=5)
    _, d, _, _ = orc.d3_ray(p2, POSE0, 0, 0)
    u, v = frame(d)
    D2, th = 5.0134, 0.0512
    s2 = Soup()
    s2.quad(D2 * d, u, v, 2.0, -d, 0)
    s2.quad((D2 + th) * d, u, v, 2.0, -d, 1)
    mats2 = [make_material(eps_r=4.0, tan_d=0.01, **WALL), make_material(pec=True, **METAL_LOBE)]
    r_plain = _scan(s2, mats2, p2)
    r_spk = _scan(s2, mats2, {**p2, "speckle": True})
    bins = {0: int(D2 / 0.01), 1: int((D2 + 2 * th) / 0.01), 2: int((D2 + 4 * th) / 0.01)}
    expect = np.zeros_like(r_spk["image"][0])
    for sg in r_plain["segments"]:
        if sg["ret_t"] > 0:
            expect[bins[int(sg["bounce"])]] += sg["ret_t"] * _speckle_direct(p2, 0, 0, int(sg["path"]),
                                                                             int(sg["bounce"]), 0)
        if sg["ret_a"] > 0:
            assert int(sg["bounce"]) == 2
            expect[bins[1]] += sg["ret_a"] * _speckle_direct(p2, 0, 0, int(sg["path"]), 2, 1)
    assert (r_plain["segments"]["ret_a"] > 0).sum() == 1
    assert np.array_equal(np.nonzero(r_spk["image"][0])[0], np.nonzero(expect)[0])
    assert np.allclose(r_spk["image"][0], expect, rtol=1e-12, atol=0.0)
    # (3) the mean over seeds: a wide wall across the beam axis, so that every
    # seed's ray (a new D3 draw) returns energy; speckled / plain per seed
    s3 = Soup()
    s3.quad((8.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0), 20.0, (-1.0, 0.0, 0.0), 0)
    wall = [make_material(eps_r=4.0, **WALL)]
    n, vals = 1500, []
    for i in range(n):
        q = {**p, "seed": 1000 + i}
        e_plain = _scan(s3, wall, q)["image"][0].sum()
        e_spk = _scan(s3, wall, {**q, "speckle": True})["image"][0].sum()
        assert e_plain > 0
        vals.append(e_spk / e_plain)
    assert abs(np.mean(vals) - 1.0) < 4.0 / math.sqrt(n), np.mean(vals)


# ----------------------------------------------------------------- termination
def check_min_energy():
    """Sec. III-A termination ("energy below detectability"): the eps_r = 4
    slab on metal at normal incidence.  The front face's reflected child
    carries E R - ret_t = (1 - W_wall(0)) / 9 (closed form).  With min_energy
    just below that energy the child is spawned (and escapes back past the
    sensor); just above it, it is not, and its energy moves from the escaped
    to the terminated tally -- by exactly that closed-form amount -- with one
    segment fewer and the same image.  min_energy = 0 spawns every child."""
    p = base_params(max_bounces=3)
    _, d, _, _ = orc.d3_ray(p, POSE0, 0, 0)
    u, v = frame(d)
    D, th = 5.0134, 0.0512
    s = Soup()
    s.quad(D * d, u, v, 2.0, -d, 0)
    s.quad((D + th) * d, u, v, 2.0, -d, 1)
    mats = [make_material(eps_r=4.0, tan_d=0.01, **WALL), make_material(pec=True, **METAL_LOBE)]
    e_child = (1.0 - scipy_window(0.6, 0.1, 30, 0.0, p["beam_width"])) / 9.0
    below = _scan(s, mats, {**p, "min_energy": e_child * (1 - 1e-4)})
    above = _scan(s, mats, {**p, "min_energy": e_child * (1 + 1e-4)})
    zero = _scan(s, mats, {**p, "min_energy": 0.0})
    tb, ta = below["tallies"][0, 0], above["tallies"][0, 0]
    assert abs((ta[3] - tb[3]) - e_child) < 1e-9 * e_child, (ta, tb, e_child)
    assert abs((tb[2] - ta[2]) - e_child) < 1e-9 * e_child
    assert ta[0] == tb[0] and ta[1] == tb[1]
    assert len(below["segments"]) == len(above["segments"]) + 1
    extra = below["segments"][(below["segments"]["bounce"] == 1) & (below["segments"]["path"] == 0)]
    assert len(extra) == 1 and extra[0]["tri"] == orc.NONE
    assert abs(extra[0]["E"] - e_child) < 1e-9 * e_child
    assert np.array_equal(below["image"], above["image"])
    # with no threshold the deeper, weaker children are spawned too
    assert len(zero["segments"]) > len(below["segments"])
    assert abs(zero["tallies"][0, 0].sum() - 1.0) < 1e-12 and abs(ta.sum() - 1.0) < 1e-12


# ----------------------------------------------------------------- range weight
def check_range_falloff():
    """The optional range weight of Eq. 1's power falloff: with exponent k a
    return at range r > 1 m is scaled by r^-k (1 m reference), so the
    normal-incidence metal plane at distance D gives W(0) D^-k; below 1 m
    nothing changes; k = 0 is the plain image; the energy tallies (physics
    of the ray tree) are unchanged."""
    p = base_params(n_bins=4000)
    _, d, _, _ = orc.d3_ray(p, POSE0, 0, 0)
    u, v = frame(d)
    mats = [make_material(pec=True, **METAL_LOBE)]
    w0 = scipy_window(0, 0, 2000, 0.0, p["beam_width"])
    for D, k in ((10.013, 4.0), (23.456, 2.0), (0.7013, 4.0)):
        s = Soup()
        s.quad(D * d, u, v, 2.0, -d, 0)
        t = plane_distance(s, 0, np.zeros(3), d)
        r = _scan(s, mats, {**p, "range_falloff": k})
        nz, e = single_return(r["image"][0])
        assert list(nz) == [int(D / p["bin_size"])]
        expect = w0 * (t ** -k if t > 1.0 else 1.0)
        assert abs(e[0] - expect) < 1e-9 * expect, (D, k, e[0], expect)
        assert abs(r["tallies"][0, 0, 0] - w0) < 1e-9 * w0
        r0 = _scan(s, mats, {**p, "range_falloff": 0.0})
        assert abs(single_return(r0["image"][0])[1][0] - w0) < 1e-9 * w0


ALL_CHECKS = [check_philox_kat, check_u24, check_d3_sigma, check_d3_pose_and_azimuth, check_fresnel_closed_forms,
              check_snell, check_brdf_normalisation, check_brdf_window_pins, check_closest_brute_force,
              check_normal_incidence_plane, check_oblique_plane, check_slab, check_slab_multipath,
              check_corner_reflector, check_lidar_like, check_conservation_tiny, check_post_pass, check_db_map,
              check_elliptic_beam, check_perlin, check_cook_torrance_lobe, check_tabulated_lobe,
              check_speckle_statistics, check_speckle_in_the_scan, check_min_energy, check_range_falloff]


@pytest.mark.parametrize("check", ALL_CHECKS, ids=lambda f: f.__name__[6:])
def test_pin(check):
    check()


def test_d3_statistics():
    check_d3_statistics()


def test_bin_returns_is_the_exactly_rounded_sum():
    """Sec. III-B binning in the oracle: each pixel equals the exact rational
    sum of its returns rounded once, whatever the order; returns past the
    last bin are dropped."""
    from fractions import Fraction
    rng = np.random.default_rng(11)
    n = 4000
    col = np.sort(rng.integers(0, 3, n)).astype(np.uint32)
    b = rng.integers(0, 6, n).astype(np.uint32)   # bin 5 lies past a 5-bin image
    e = (10.0 ** rng.uniform(-9, 0, n)).astype(np.float32)
    out = orc.bin_returns(col, b, e, 3, 5)
    for c in range(3):
        for k in range(5):
            sel = (col == c) & (b == k)
            exact = sum((Fraction(float(x)) for x in e[sel]), Fraction(0))
            assert out[c, k] == float(exact)
    # a cancelling sum that naive left-to-right addition gets wrong
    vals = np.array([1e16, 1.0, -1e16, 1.0], np.float64)
    assert orc.bin_returns(np.zeros(4, np.uint32), np.zeros(4, np.uint32), vals, 1, 1)[0, 0] == 2.0


def test_ray_stride_traces_exactly_the_sampled_rays():
    """A sample of every s-th initial ray of a column traces those rays as the
    full scan does (each initial ray's tree depends only on its own counter):
    the same segments and tallies for them, nothing for the others, and the
    sample's image is the full scan's image of those rays alone."""
    from paper_2310_03505_gb300 import scenes
    sc, pz, s = scenes.config_tiny()
    cols = [3, 77, 200, 391]
    full = orc.scan(sc.vertices, sc.triangles, sc.material_ids, sc.materials, pz, s, az_list=cols, post=False)
    stride = 3
    part = orc.scan(sc.vertices, sc.triangles, sc.material_ids, sc.materials, pz, {**s, "ray_stride": stride},
                    az_list=cols, post=False)
    keep = np.arange(s["rays_per_beam"]) % stride == 0
    assert np.array_equal(part["tallies"][:, keep], full["tallies"][:, keep])
    assert not part["tallies"][:, ~keep].any() and not part["flags"][:, ~keep].any()
    fs = full["segments"][full["segments"]["k"] % stride == 0]
    ps = part["segments"]
    assert len(ps) == len(fs) > 0
    key = lambda a: np.lexsort((a["path"], a["bounce"], a["k"], a["az"]))
    assert np.array_equal(ps[key(ps)], fs[key(fs)])
    # a stride of the whole beam traces ray 0 alone: the image holds at most its returned energy
    one = orc.scan(sc.vertices, sc.triangles, sc.material_ids, sc.materials, pz,
                   {**s, "ray_stride": s["rays_per_beam"]}, az_list=[77], post=False)
    assert not one["tallies"][0, 1:].any()
    assert 0 < one["image"].sum() <= one["tallies"][0, 0, 0] * (1 + 1e-12)
