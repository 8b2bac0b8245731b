"""Seeded synthetic inputs: triangle scenes, sensor settings and poses.

This module holds inputs only -- geometry, material tables and sensor
settings -- and none of the simulator's arithmetic.  It is the one module
that both the CUDA path and the FP64 oracle are fed from.

The paper's own workloads are reconstructed meshes of the MulRan DCC/KAIST
sequences (8.8M and 12.4M triangles, Sec. IV-A) driven with 400 azimuths,
D3 beams of b = 10 deg at P = 90 % and at most 4 reflections (Sec. IV).  Those
meshes are not available, so procedural scenes of the same kind stand in:

* ``tiny_room``   -- 10 x 10 x 3 m room (1,664 triangles) with 20 seeded
  axis-aligned cubes (240 triangles), two materials.
* ``campus``      -- about 200k triangles: gridded ground, 200 extruded
  buildings, 500 closed cylinders, six materials.
* ``city``        -- about 5M triangles: a gridded street block pattern of
  buildings with window-glass panels, parked cars and lamp poles.

Every generator is deterministic for a given seed (numpy PCG64).  Triangles
are wound so that the geometric normal (v1 - v0) x (v2 - v0) points out of
the triangle's material; room walls are single sheets whose normals face the
room, the ground is a single sheet facing up.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# material presets
# --------------------------------------------------------------------------
# BRDF parameters (A, B, C) of Eq. 5 with S = 1 - A - B.  The tuples fitted in
# Sec. IV-B are printed as (v, A, S, C); B is recovered as 1 - A - S.  The
# metal tuple (A, S) = (1.0, 1.0) violates A + B <= 1 and is read as a pure
# specular lobe A = B = 0, S = 1, C = 2000.
BRDF_PRESETS = {
    "wall": dict(A=0.6, B=0.1, C=30.0),
    "wood": dict(A=0.6, B=0.1, C=70.0),
    "glass": dict(A=0.01, B=0.95, C=1900.0),
    "metal": dict(A=0.0, B=0.0, C=2000.0),
}


def material(eps_r=1.0, loss_tangent=0.0, brdf="wall", pec=False, name=""):
    b = BRDF_PRESETS[brdf]
    return dict(name=name, eps_r=float(eps_r), loss_tangent=float(loss_tangent),
                A=b["A"], B=b["B"], C=b["C"], pec=bool(pec))


# relative permittivity and loss tangent of the synthetic materials (proposed;
# the configurations only bound eps_r to 1..10)
def cook_torrance(eps_r, loss_tangent, diffuse, roughness, name=""):
    """A material with the Cook-Torrance lobe (diffuse amount, Beckmann
    roughness; the paper's setting in Sec. IV is diffuse 0.2, roughness 0.5).
    Its Fresnel split and losses come from eps_r and the loss tangent as for
    every material."""
    return dict(name=name, eps_r=float(eps_r), loss_tangent=float(loss_tangent), A=float(diffuse),
                B=float(roughness), C=0.0, pec=False, lobe="cook_torrance")


LOBE_SAMPLES = 4097


def tabulated(eps_r, loss_tangent, density, name=""):
    """A material with a user lobe: density(x) sampled at the 4097 points
    x_j = j (pi/2) / 4096 of [0, pi/2] (float32)."""
    x = np.arange(LOBE_SAMPLES) * (0.5 * math.pi / (LOBE_SAMPLES - 1))
    t = np.asarray(density(x), np.float32).astype(np.float64)
    return dict(name=name, eps_r=float(eps_r), loss_tangent=float(loss_tangent), A=0.6, B=0.1, C=30.0, pec=False,
                lobe="table", lobe_table=t)


MATERIALS = {
    "metal": material(pec=True, brdf="metal", name="metal"),
    "dielectric": material(4.0, 0.01, "wall", name="dielectric"),
    "concrete": material(5.3, 0.05, "wall", name="concrete"),
    "glass": material(6.3, 0.02, "glass", name="glass"),
    "wood": material(2.0, 0.05, "wood", name="wood"),
    "vegetation": material(1.5, 0.3, "wall", name="vegetation"),
    "asphalt": material(3.2, 0.03, "wall", name="asphalt"),
    "brick": material(4.5, 0.04, "wall", name="brick"),
    "plastic": material(2.5, 0.01, "wood", name="plastic"),
}


@dataclass
class Scene:
    name: str
    vertices: np.ndarray        # float32 [V, 3]
    triangles: np.ndarray       # uint32  [T, 3]
    material_ids: np.ndarray    # uint16  [T]
    materials: list = field(default_factory=list)   # dicts, see material()
    # axis-aligned boxes (lo, hi) of the solid objects, for placing sensors
    obstacles: list = field(default_factory=list)

    @property
    def n_triangles(self) -> int:
        return int(self.triangles.shape[0])


class _Mesh:
    """Triangle soup builder with outward-normal enforcement."""

    def __init__(self):
        self.v = []
        self.t = []
        self.m = []
        self.nv = 0

    def _add_tri(self, a, b, c, normal, mat):
        a = np.asarray(a, np.float64)
        b = np.asarray(b, np.float64)
        c = np.asarray(c, np.float64)
        if np.dot(np.cross(b - a, c - a), normal) < 0:
            b, c = c, b
        self.v.extend([a, b, c])
        self.t.append((self.nv, self.nv + 1, self.nv + 2))
        self.m.append(mat)
        self.nv += 3

    def quad_grid(self, origin, eu, ev, nu, nv, normal, mat):
        """Grid of nu x nv cells over the parallelogram origin + s*eu + t*ev."""
        origin = np.asarray(origin, np.float64)
        eu = np.asarray(eu, np.float64)
        ev = np.asarray(ev, np.float64)
        normal = np.asarray(normal, np.float64)
        base = self.nv
        P = np.empty(((nu + 1) * (nv + 1), 3))
        for j in range(nv + 1):
            for i in range(nu + 1):
                P[j * (nu + 1) + i] = origin + eu * (i / nu) + ev * (j / nv)
        self.v.extend(list(P))
        self.nv += P.shape[0]
        flip = np.dot(np.cross(eu, ev), normal) < 0
        for j in range(nv):
            for i in range(nu):
                p00 = base + j * (nu + 1) + i
                p10 = p00 + 1
                p01 = p00 + (nu + 1)
                p11 = p01 + 1
                tris = ((p00, p10, p11), (p00, p11, p01))
                for a, b, c in tris:
                    self.t.append((a, c, b) if flip else (a, b, c))
                    self.m.append(mat)

    def box(self, lo, hi, mat, cell=None, skip_bottom=False):
        """Closed axis-aligned box, outward normals, optional facade grid."""
        lo = np.asarray(lo, np.float64)
        hi = np.asarray(hi, np.float64)
        ext = hi - lo

        def n(length):
            return 1 if cell is None else max(1, int(math.ceil(length / cell)))

        x0, y0, z0 = lo
        x1, y1, z1 = hi
        ex, ey, ez = np.eye(3)
        # -x, +x
        self.quad_grid((x0, y0, z0), ey * ext[1], ez * ext[2], n(ext[1]), n(ext[2]), -ex, mat)
        self.quad_grid((x1, y0, z0), ey * ext[1], ez * ext[2], n(ext[1]), n(ext[2]), ex, mat)
        # -y, +y
        self.quad_grid((x0, y0, z0), ex * ext[0], ez * ext[2], n(ext[0]), n(ext[2]), -ey, mat)
        self.quad_grid((x0, y1, z0), ex * ext[0], ez * ext[2], n(ext[0]), n(ext[2]), ey, mat)
        # bottom, top
        if not skip_bottom:
            self.quad_grid((x0, y0, z0), ex * ext[0], ey * ext[1], 1, 1, -ez, mat)
        self.quad_grid((x0, y0, z1), ex * ext[0], ey * ext[1], n(ext[0]), n(ext[1]), ez, mat)

    def cylinder(self, cx, cy, z0, z1, r, seg, mat):
        """Closed cylinder: seg side quads and two triangle-fan caps."""
        ang = np.arange(seg) * (2 * np.pi / seg)
        ring = np.stack([cx + r * np.cos(ang), cy + r * np.sin(ang)], 1)
        for i in range(seg):
            a = ring[i]
            b = ring[(i + 1) % seg]
            mid = 0.5 * (a + b)
            nrm = np.array([mid[0] - cx, mid[1] - cy, 0.0])
            p00 = (a[0], a[1], z0)
            p10 = (b[0], b[1], z0)
            p11 = (b[0], b[1], z1)
            p01 = (a[0], a[1], z1)
            self._add_tri(p00, p10, p11, nrm, mat)
            self._add_tri(p00, p11, p01, nrm, mat)
            self._add_tri((cx, cy, z1), p01, p11, (0, 0, 1), mat)
            self._add_tri((cx, cy, z0), p10, p00, (0, 0, -1), mat)

    def build(self, name, materials) -> Scene:
        v = np.asarray(self.v, np.float64).astype(np.float32)
        t = np.asarray(self.t, np.uint32).reshape(-1, 3)
        m = np.asarray(self.m, np.uint16)
        return Scene(name, v, t, m, materials)


def _aabb_gap(lo_a, hi_a, lo_b, hi_b):
    """Largest per-axis separation between two boxes (negative: overlap)."""
    return max(float(np.max(lo_b - hi_a)), float(np.max(lo_a - hi_b)))


def _point_box_dist(p, lo, hi):
    q = np.clip(p, lo, hi)
    return float(np.linalg.norm(p - q))


# --------------------------------------------------------------------------
# tiny room
# --------------------------------------------------------------------------
def tiny_room(seed: int = 0x5EED0000, n_cubes: int = 20) -> Scene:
    """10 x 10 x 3 m room (floor/ceiling 16 x 16 grids, walls 16 x 5 grids)
    with n_cubes non-overlapping axis-aligned cubes, side U(0.3, 1.5) m, at
    least 1 m from the sensor at (0, 0, 0.5).  Material 0 is a perfect
    conductor, material 1 a dielectric (eps_r = 4, tan delta = 0.01); the room
    is material 1 and the cubes alternate, starting from a seeded choice."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mesh = _Mesh()
    L, H = 5.0, 3.0
    room_mat = 1
    # floor (normal +z into the room), ceiling (-z)
    mesh.quad_grid((-L, -L, 0.0), (2 * L, 0, 0), (0, 2 * L, 0), 16, 16, (0, 0, 1), room_mat)
    mesh.quad_grid((-L, -L, H), (2 * L, 0, 0), (0, 2 * L, 0), 16, 16, (0, 0, -1), room_mat)
    # walls, normals into the room
    mesh.quad_grid((-L, -L, 0.0), (0, 2 * L, 0), (0, 0, H), 16, 5, (1, 0, 0), room_mat)
    mesh.quad_grid((L, -L, 0.0), (0, 2 * L, 0), (0, 0, H), 16, 5, (-1, 0, 0), room_mat)
    mesh.quad_grid((-L, -L, 0.0), (2 * L, 0, 0), (0, 0, H), 16, 5, (0, 1, 0), room_mat)
    mesh.quad_grid((-L, L, 0.0), (2 * L, 0, 0), (0, 0, H), 16, 5, (0, -1, 0), room_mat)
    sensor = np.array([0.0, 0.0, 0.5])
    boxes = []
    first = int(rng.integers(0, 2))
    tries = 0
    while len(boxes) < n_cubes:
        tries += 1
        if tries > 100000:
            raise RuntimeError("cube placement failed")
        s = rng.uniform(0.3, 1.5)
        h = s / 2 + 0.05
        c = np.array([rng.uniform(-L + h, L - h), rng.uniform(-L + h, L - h), rng.uniform(h, H - h)])
        lo, hi = c - s / 2, c + s / 2
        if _point_box_dist(sensor, lo, hi) < 1.0:
            continue
        if any(_aabb_gap(lo, hi, blo, bhi) < 0.05 for blo, bhi in boxes):
            continue
        boxes.append((lo, hi))
    for i, (lo, hi) in enumerate(boxes):
        mesh.box(lo, hi, (first + i) % 2)
    mats = [MATERIALS["metal"], MATERIALS["dielectric"]]
    return mesh.build("tiny_room", mats)


# --------------------------------------------------------------------------
# campus
# --------------------------------------------------------------------------
CAMPUS_MATS = ["metal", "concrete", "glass", "wood", "vegetation", "asphalt"]


def campus(seed: int = 0x5EED0001, target_tris: int = 200_000, n_buildings: int = 200,
           n_cylinders: int = 500, extent: float = 150.0) -> Scene:
    """Procedural campus: a gridded 300 x 300 m ground sheet (asphalt), n_buildings
    non-overlapping closed boxes (footprint U(5, 20) m, height U(5, 30) m,
    facades gridded to about 3 m, sunk 0.5 m into the ground) and n_cylinders
    closed 16-segment cylinders (radius U(0.2, 0.5) m).  The ground grid is
    sized so that the total triangle count lands within 5 % of target_tris."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mesh = _Mesh()
    idx = {n: i for i, n in enumerate(CAMPUS_MATS)}
    sensor = np.array([0.0, 0.0, 1.8])
    boxes = []
    tries = 0
    while len(boxes) < n_buildings:
        tries += 1
        if tries > 200000:
            raise RuntimeError("building placement failed")
        w, d = rng.uniform(5, 20, size=2)
        h = rng.uniform(5, 30)
        cx, cy = rng.uniform(-extent + 2 + w / 2, extent - 2 - w / 2), rng.uniform(-extent + 2 + d / 2, extent - 2 - d / 2)
        lo = np.array([cx - w / 2, cy - d / 2, -0.5])
        hi = np.array([cx + w / 2, cy + d / 2, h])
        if _point_box_dist(sensor, lo, hi) < 10.0:
            continue
        if any(_aabb_gap(lo, hi, blo, bhi) < 1.0 for blo, bhi, _ in boxes):
            continue
        u = rng.uniform()
        mat = "concrete" if u < 0.5 else "glass" if u < 0.7 else "metal" if u < 0.85 else "wood"
        boxes.append((lo, hi, mat))
    for lo, hi, mat in boxes:
        mesh.box(lo, hi, idx[mat], cell=3.0)
    cyl = []
    tries = 0
    while len(cyl) < n_cylinders:
        tries += 1
        if tries > 500000:
            raise RuntimeError("cylinder placement failed")
        r = rng.uniform(0.2, 0.5)
        x, y = rng.uniform(-extent + 1, extent - 1, size=2)
        hgt = rng.uniform(3.0, 10.0)
        lo = np.array([x - r, y - r, -0.2])
        hi = np.array([x + r, y + r, hgt])
        if _point_box_dist(sensor, lo, hi) < 3.0:
            continue
        if any(_aabb_gap(lo, hi, blo, bhi) < 0.5 for blo, bhi, _ in boxes):
            continue
        if any(_aabb_gap(lo, hi, clo, chi) < 0.3 for clo, chi in cyl):
            continue
        cyl.append((lo, hi))
        mat = "metal" if rng.uniform() < 0.5 else "vegetation"
        mesh.cylinder(x, y, -0.2, hgt, r, 16, idx[mat])
    others = len(mesh.t)
    g = max(1, int(round(math.sqrt(max(target_tris - others, 2) / 2.0))))
    mesh.quad_grid((-extent, -extent, 0.0), (2 * extent, 0, 0), (0, 2 * extent, 0), g, g, (0, 0, 1), idx["asphalt"])
    mats = [MATERIALS[n] for n in CAMPUS_MATS]
    sc = mesh.build("campus", mats)
    sc.obstacles = [(lo, hi) for lo, hi, _ in boxes] + list(cyl)
    return sc


def _free(foot, x, y, clearance, extent):
    if abs(x) > extent or abs(y) > extent:
        return False
    if not len(foot):
        return True
    inside = ((x > foot[:, 0] - clearance) & (x < foot[:, 2] + clearance) &
              (y > foot[:, 1] - clearance) & (y < foot[:, 3] + clearance))
    return not bool(inside.any())


def _footprints(sc: Scene) -> np.ndarray:
    return np.array([[lo[0], lo[1], hi[0], hi[1]] for lo, hi in sc.obstacles], np.float64).reshape(-1, 4)


def random_pose(sc: Scene, rng, height: float = 1.8, extent: float = 100.0, clearance: float = 1.0) -> dict:
    """A seeded sensor pose uniform over [-extent, extent]^2 at the given
    height, clear of every obstacle footprint, with a uniform heading."""
    foot = _footprints(sc)
    for _ in range(10000):
        x, y = (float(v) for v in rng.uniform(-extent, extent, size=2))
        if _free(foot, x, y, clearance, extent):
            return pose(x, y, height, yaw=float(rng.uniform(-math.pi, math.pi)))
    raise RuntimeError("no free sensor position found")


def trajectory(sc: Scene, n: int, step: float = 0.25, seed: int = 0x5EED0003, height: float = 1.8,
               turn_sigma_deg: float = 10.0, clearance: float = 1.0, extent: float = 140.0) -> list:
    """Seeded random walk of n sensor poses, step metres apart: the heading
    changes by N(0, turn_sigma) per step; a step that would come within
    clearance of an obstacle's footprint or leave [-extent, extent]^2 is
    redrawn with a fresh heading.  Starts at the origin (kept clear of
    obstacles by the generators)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    foot = _footprints(sc)

    def free(x, y):
        return _free(foot, x, y, clearance, extent)

    x, y = 0.0, 0.0
    heading = float(rng.uniform(-math.pi, math.pi))
    out = []
    for _ in range(n):
        out.append(pose(x, y, height, yaw=heading))
        for attempt in range(1000):
            h = heading + math.radians(turn_sigma_deg) * float(rng.standard_normal()) if attempt == 0 else \
                float(rng.uniform(-math.pi, math.pi))
            nx, ny = x + step * math.cos(h), y + step * math.sin(h)
            if free(nx, ny):
                x, y, heading = nx, ny, h
                break
    return out


# --------------------------------------------------------------------------
# city (large)
# --------------------------------------------------------------------------
CITY_MATS = ["metal", "concrete", "glass", "wood", "vegetation", "asphalt", "brick", "plastic"]


def city(seed: int = 0x5EED0002, target_tris: int = 5_000_000, blocks: int = 12, extent: float = 300.0) -> Scene:
    """Procedural city of about target_tris triangles: a blocks x blocks street
    grid of building lots (brick/concrete facades gridded to about 1.5 m with
    inset window-glass panels), parked-car boxes along the streets and
    lamp-pole cylinders; a gridded asphalt ground fills the rest of the
    triangle budget.  Eight materials."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mesh = _Mesh()
    idx = {n: i for i, n in enumerate(CITY_MATS)}
    lot = 2 * extent / blocks
    street = 14.0
    obstacles = []
    for bi in range(blocks):
        for bj in range(blocks):
            x0 = -extent + bi * lot + street / 2
            y0 = -extent + bj * lot + street / 2
            size = lot - street
            if abs(x0 + size / 2) < lot / 2 and abs(y0 + size / 2) < lot / 2:
                continue  # the sensor's plaza
            # split the lot into 2x2 buildings
            for si in range(2):
                for sj in range(2):
                    w = size / 2 - 2.0
                    lo = np.array([x0 + si * size / 2 + 1.0, y0 + sj * size / 2 + 1.0, -0.5])
                    h = rng.uniform(8, 45)
                    hi = lo + np.array([w, w, h + 0.5])
                    mat = "brick" if rng.uniform() < 0.5 else "concrete"
                    mesh.box(lo, hi, idx[mat], cell=1.5)
                    obstacles.append((lo.copy(), hi.copy()))
                    # glass panels 5 cm in front of the +x / -x facades
                    for side in (0, 1):
                        xf = hi[0] + 0.05 if side else lo[0] - 0.05
                        nrm = (1, 0, 0) if side else (-1, 0, 0)
                        nwin = int(w // 4)
                        nfl = int(h // 4)
                        for a in range(nwin):
                            for f in range(nfl):
                                y = lo[1] + 1.0 + a * 4.0
                                z = 1.0 + f * 4.0
                                mesh.quad_grid((xf, y, z), (0, 2.0, 0), (0, 0, 2.0), 1, 1, nrm, idx["glass"])
            # parked cars and poles along the lot's south street
            for c in range(int(size // 6)):
                cx = x0 + 3 + c * 6
                cy = y0 - 3.0
                lo = np.array([cx - 2.2, cy - 0.9, 0.15])
                hi = np.array([cx + 2.2, cy + 0.9, 1.5])
                mesh.box(lo, hi, idx["metal" if rng.uniform() < 0.7 else "plastic"])
                obstacles.append((lo, hi))
            for c in range(int(size // 20)):
                mesh.cylinder(x0 + 10 + c * 20, y0 - 5.5, -0.2, 6.0, 0.12, 16, idx["metal"])
                px, py = x0 + 10 + c * 20, y0 - 5.5
                obstacles.append((np.array([px - 0.12, py - 0.12, -0.2]), np.array([px + 0.12, py + 0.12, 6.0])))
    others = len(mesh.t)
    g = max(1, int(round(math.sqrt(max(target_tris - others, 2) / 2.0))))
    mesh.quad_grid((-extent, -extent, 0.0), (2 * extent, 0, 0), (0, 2 * extent, 0), g, g, (0, 0, 1), idx["asphalt"])
    mats = [MATERIALS[n] for n in CITY_MATS]
    sc = mesh.build("city", mats)
    sc.obstacles = obstacles
    return sc


# --------------------------------------------------------------------------
# sensor settings and poses
# --------------------------------------------------------------------------
def f32(x) -> float:
    """Round to the nearest float32 so that both implementations read the same number."""
    return float(np.float32(x))


def sensor(**kw) -> dict:
    """Sensor settings with the paper's defaults (Sec. IV): 400 azimuths,
    50 rays per beam, D3 with b = 10 deg and P = 0.9, at most 4 reflections."""
    p = dict(n_azimuth=400, rays_per_beam=50, max_bounces=4, n_bins=1142,
             beam_width=math.radians(10.0), beam_prob=0.9, elevation=0.0, bin_size=0.0438,
             t_min=1e-4, min_energy=0.0, freq_hz=76.5e9, blur_sigma_bins=0.0, az_pattern_sigma=0.0,
             noise_sys=0.0, noise_amb=0.0, multipath=True, refraction=True, speckle=False, noise=False,
             perlin=False, beam_aspect=1.0, noise_cell_az=8.0, noise_cell_bins=32.0, range_falloff=0.0,
             seed=0x5EED, scan_id=0)
    p.update(kw)
    for k in ("beam_width", "beam_prob", "elevation", "bin_size", "t_min", "min_energy", "freq_hz",
              "blur_sigma_bins", "az_pattern_sigma", "noise_sys", "noise_amb", "beam_aspect", "noise_cell_az",
              "noise_cell_bins", "range_falloff"):
        p[k] = f32(p[k])
    for k in ("n_azimuth", "rays_per_beam", "max_bounces", "n_bins", "seed", "scan_id"):
        p[k] = int(p[k])
    return p


# Beam width of the tiny configuration: a D3 radius with sigma = 0.9 deg at
# P = 0.9 corresponds to b = 2 * 0.9 deg * 1.6448536 = 2.9607365 deg.
TINY_BEAM_WIDTH_DEG = 2.960736528512652


def pose(x=0.0, y=0.0, z=0.0, yaw=0.0) -> dict:
    return dict(p=(f32(x), f32(y), f32(z)), q=(f32(math.cos(yaw / 2)), 0.0, 0.0, f32(math.sin(yaw / 2))))


# the workload configurations ------------------------------------------------
def config_tiny(**kw):
    """Tiny plain scan: room + 20 cubes, 400 x 8 rays, sigma = 0.9 deg, <= 3
    bounces, 1142 bins x 0.0438 m (50 m)."""
    s = sensor(n_azimuth=400, rays_per_beam=8, max_bounces=3, n_bins=1142, bin_size=0.0438,
               beam_width=math.radians(TINY_BEAM_WIDTH_DEG), **kw)
    return tiny_room(), pose(0.0, 0.0, 0.5), s


def config_medium(**kw):
    """Medium plain scan: ~200k-triangle campus, 400 x 200 rays, D3 b = 10 deg,
    <= 5 bounces, refraction on, 2000 bins to 87.6 m."""
    s = sensor(n_azimuth=400, rays_per_beam=200, max_bounces=5, n_bins=2000, bin_size=0.0438,
               beam_width=math.radians(10.0), **kw)
    return campus(), pose(0.0, 0.0, 1.8), s


def config_batched(n_scans: int = 256, seed: int = 0x5EED0003, **kw):
    """Batched scans: n_scans poses every 0.25 m along a seeded random walk
    through a ~1M-triangle scene of the campus generator, 400 beams each with
    rays per beam drawn uniformly from {32, ..., 512} per pose; otherwise the
    medium sensor (<= 5 bounces, refraction on, 2000 bins to 87.6 m).
    Returns (scene, poses, params)."""
    sc = campus(target_tris=1_000_000)
    poses = trajectory(sc, n_scans, step=0.25, seed=seed)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    ns = rng.integers(32, 513, size=n_scans)
    params = [sensor(n_azimuth=400, rays_per_beam=int(ns[i]), max_bounces=5, n_bins=2000, bin_size=0.0438,
                     beam_width=math.radians(10.0), scan_id=i, **kw) for i in range(n_scans)]
    return sc, poses, params


def config_large(**kw):
    """Large plain scan: ~5M-triangle city, 400 x 1000 rays, <= 8 bounces,
    4000 bins x 0.04375 m (175 m)."""
    s = sensor(n_azimuth=400, rays_per_beam=1000, max_bounces=8, n_bins=4000, bin_size=0.04375,
               beam_width=math.radians(10.0), **kw)
    return city(), pose(0.0, 0.0, 1.8), s
