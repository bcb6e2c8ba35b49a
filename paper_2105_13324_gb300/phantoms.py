"""Seeded synthetic inputs: phantoms, acquisition geometries and Poisson noise.

This module produces inputs only.  It holds none of the transport or
reconstruction arithmetic, and both the CUDA path and the CPU oracle consume
what it makes.

The paper (Sec. 5.4-5.5) evaluates on MCAT/XCAT torsos, physical thorax
phantoms and patients, none of which are available; these seeded phantoms
stand in for them with the same structure: a water cylinder with an
ellipsoidal myocardial shell, and a torso with lungs, spine, liver and a
heart shell carrying a transmural defect.  Acquisition follows Sec. 3:
one parallel-hole collimated head per view, views rotating over 180 or 360
degrees around the body axis z.

Conventions (shared input contract):
  * grid centred on the origin, x fastest: ``material[z, y, x]`` (uint8 index
    into the material table);
  * material table rows: density rho (g/cm^3), electrons per nucleon Z/A, and
    effective atomic number Z_eff;
  * distances in mm, energies in keV, angles in degrees.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Material table rows (rho g/cm^3, Z/A, Z_eff).
AIR = (0.001205, 0.4992, 7.64)
WATER = (1.0, 0.55509, 7.42)
SOFT_TISSUE = (1.0, 0.5494, 7.42)
LUNG = (0.3, 0.5494, 7.42)
BONE = (1.85, 0.5148, 13.0)

# Photoelectric coefficient k of the attenuation model mu = rho (N_A Z/A
# sigma_KN(E) + k Z_eff^4 / E^3): chosen so that water has mu = 0.154 /cm at
# 140.5 keV (the stated attenuation of the 32^3 water-cylinder workload).
PHOTO_K = 2.70259

TC99M_KEV = 140.5


@dataclass
class Phantom:
    """A voxelised attenuation map plus the activity used to make data."""

    material: np.ndarray          # uint8 [nz, ny, nx]
    rho: np.ndarray               # float64 [n_materials]
    z_over_a: np.ndarray          # float64 [n_materials]
    z_eff: np.ndarray             # float64 [n_materials]
    voxel_mm: float
    activity: np.ndarray | None = None  # float32 [nz, ny, nx]
    labels: dict = field(default_factory=dict)  # name -> bool mask (fixtures)

    @property
    def shape(self):
        return self.material.shape

    @property
    def n_voxels(self) -> int:
        return int(self.material.size)


@dataclass
class Geometry:
    """Acquisition geometry of a parallel-hole SPECT camera (Sec. 3)."""

    n_views: int
    arc_deg: float
    n_bins_u: int
    n_bins_v: int
    bin_mm: float
    radius_mm: float
    start_deg: float = 0.0
    hole_len_mm: float = 35.0
    hole_diam_mm: float = 1.5
    fwhm_mm: float = 3.5
    e0_kev: float = TC99M_KEV
    window_frac: float = 0.20
    photo_k: float = PHOTO_K

    @property
    def n_rows(self) -> int:
        return self.n_views * self.n_bins_u * self.n_bins_v


def _table(rows):
    a = np.asarray(rows, dtype=np.float64)
    return a[:, 0].copy(), a[:, 1].copy(), a[:, 2].copy()


def voxel_centres(n: int, h: float) -> np.ndarray:
    """Centres of n voxels of size h on a grid centred on the origin."""
    return (np.arange(n, dtype=np.float64) + 0.5) * h - 0.5 * n * h


def front_face_radius(n_xy: int, h: float) -> float:
    """Collimator front face: 10 mm beyond the half-diagonal of the grid."""
    return math.sqrt(0.5) * n_xy * h + 10.0


def _grid(n, h):
    c = voxel_centres(n, h)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    return x, y, z


def _ellipsoid(x, y, z, c, a):
    return ((x - c[0]) / a[0]) ** 2 + ((y - c[1]) / a[1]) ** 2 + ((z - c[2]) / a[2]) ** 2 <= 1.0


def water_cylinder_phantom(n: int = 32, h: float = 4.0, radius: float = 50.0,
                           shell_outer=(24.0, 20.0, 20.0), wall: float = 8.0,
                           shell_activity: float = 4.0) -> Phantom:
    """Water cylinder (axis z) in air with an ellipsoidal shell source.

    Materials: 0 = air, 1 = water.  Activity: shell 4, water 1, air 0.
    """
    x, y, z = _grid(n, h)
    cyl = x * x + y * y <= radius * radius
    outer = _ellipsoid(x, y, z, (0, 0, 0), shell_outer)
    inner = _ellipsoid(x, y, z, (0, 0, 0), tuple(s - wall for s in shell_outer))
    shell = outer & ~inner
    mat = np.zeros((n, n, n), np.uint8)
    mat[cyl] = 1
    act = np.zeros((n, n, n), np.float32)
    act[cyl] = 1.0
    act[shell] = shell_activity
    rho, zoa, zeff = _table([AIR, WATER])
    return Phantom(mat, rho, zoa, zeff, h, act, {"body": cyl, "shell": shell})


def torso_phantom(n: int = 64, h: float = 3.2, seed: int | None = None,
                  heart_centre=(25.0, 20.0, 0.0), heart_outer=(20.0, 20.0, 24.0),
                  wall: float = 8.0, defect_deg: float = 90.0, defect_width_deg: float = 45.0,
                  defect_uptake: float = 0.5, scale_jitter: float = 0.10) -> Phantom:
    """Cardiac torso: elliptic body, two lungs, spine, liver, heart shell.

    Materials: 0 = air, 1 = soft tissue, 2 = lung, 3 = bone.
    Activity: heart 4 (defect sector x defect_uptake), liver 2, lungs 0.5,
    rest of the body 1.  With ``seed`` set, each organ semi-axis is scaled by
    1 + scale_jitter*(2u - 1), u uniform from numpy's Philox generator.
    The body (300 x 200 mm) is clipped by grids narrower than 300 mm.
    """
    rng = np.random.Generator(np.random.Philox(seed)) if seed is not None else None

    def jit(a):
        if rng is None:
            return tuple(float(v) for v in a)
        return tuple(float(v) * (1.0 + scale_jitter * (2.0 * rng.random() - 1.0)) for v in a)

    x, y, z = _grid(n, h)
    body_ax = jit((150.0, 100.0))
    lung_ax = jit((45.0, 60.0, 90.0))
    spine_r = jit((15.0,))[0]
    liver_ax = jit((70.0, 60.0, 45.0))
    heart_ax = jit(heart_outer)
    body = (x / body_ax[0]) ** 2 + (y / body_ax[1]) ** 2 <= 1.0
    lung_l = _ellipsoid(x, y, z, (70.0, 10.0, 20.0), lung_ax)
    lung_r = _ellipsoid(x, y, z, (-70.0, 10.0, 20.0), lung_ax)
    lungs = (lung_l | lung_r) & body
    spine = ((x - 0.0) ** 2 + (y + 75.0) ** 2 <= spine_r * spine_r) & body
    liver = _ellipsoid(x, y, z, (-55.0, -10.0, -70.0), liver_ax) & body
    h_out = _ellipsoid(x, y, z, heart_centre, heart_ax)
    h_in = _ellipsoid(x, y, z, heart_centre, tuple(max(s - wall, 1e-3) for s in heart_ax))
    heart = h_out & ~h_in & body
    ang = np.degrees(np.arctan2(y - heart_centre[1], x - heart_centre[0]))
    dang = (ang - defect_deg + 180.0) % 360.0 - 180.0
    defect = heart & (np.abs(dang) <= 0.5 * defect_width_deg)

    mat = np.zeros((n, n, n), np.uint8)
    mat[body] = 1
    mat[lungs] = 2
    mat[spine] = 3
    act = np.zeros((n, n, n), np.float32)
    act[body] = 1.0
    act[lungs] = 0.5
    act[liver] = 2.0
    act[heart] = 4.0
    act[defect] = 4.0 * defect_uptake
    rho, zoa, zeff = _table([AIR, SOFT_TISSUE, LUNG, BONE])
    labels = {"body": body, "lungs": lungs, "spine": spine, "liver": liver, "heart": heart,
              "defect": defect, "heart_centre": np.asarray(heart_centre)}
    return Phantom(mat, rho, zoa, zeff, h, act, labels)


def slab_phantom(n: int, h: float, material_row, thickness_mm: float, extra_rows=()) -> Phantom:
    """A slab of one material, perpendicular to x, centred on the origin.

    Voxels with |x| < thickness/2 hold material 1; the rest is material 0,
    a vacuum row (rho = 0).  ``extra_rows`` appends table rows that are not
    used in the map (they still enter the majorant).
    """
    c = voxel_centres(n, h)
    mat = np.zeros((n, n, n), np.uint8)
    mat[:, :, np.abs(c) < 0.5 * thickness_mm] = 1
    rho, zoa, zeff = _table([(0.0, 0.5, 7.0), material_row, *extra_rows])
    return Phantom(mat, rho, zoa, zeff, h)


def vacuum_phantom(n: int, h: float) -> Phantom:
    """A grid whose only material has rho = 0 (nothing attenuates)."""
    mat = np.zeros((n, n, n), np.uint8)
    rho, zoa, zeff = _table([(0.0, 0.5, 7.0)])
    return Phantom(mat, rho, zoa, zeff, h, np.ones((n, n, n), np.float32))


def uniform_phantom(n: int, h: float, material_row=WATER) -> Phantom:
    mat = np.ones((n, n, n), np.uint8)
    rho, zoa, zeff = _table([AIR, material_row])
    return Phantom(mat, rho, zoa, zeff, h, np.ones((n, n, n), np.float32))


def spect_geometry(n_views: int, arc_deg: float, n_bins: int, bin_mm: float, n_xy: int,
                   voxel_mm: float, **kw) -> Geometry:
    return Geometry(n_views=n_views, arc_deg=arc_deg, n_bins_u=n_bins, n_bins_v=n_bins,
                    bin_mm=bin_mm, radius_mm=front_face_radius(n_xy, voxel_mm), **kw)


# --------------------------------------------------------------------------
# The five workloads
# --------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    phantom: Phantom
    geometry: Geometry
    n_histories: int
    seed: int
    mlem_iters: int
    total_counts: float
    noise_seed: int


def workload(name: str) -> Workload:
    """Named workloads.

    ``water32``: 32^3 x 4 mm water cylinder, 16 views / 180 deg, 32^2 x 4 mm
    bins, 2e6 histories (seed 1), 20 MLEM iterations, 1e6 counts.
    ``torso64``: 64^3 x 3.2 mm torso, 60 views / 180 deg, 64^2 x 3.2 mm bins,
    1e8 histories, 50 MLEM iterations, 5e6 counts (noise seed 2).
    ``torso128``: 128^3 x 2 mm torso with organ sizes jittered +-10 % (seed 3),
    120 views / 360 deg, 128^2 x 2 mm bins, 1e9 histories, 50 iterations,
    2e7 counts.
    """
    if name == "water32":
        ph = water_cylinder_phantom()
        g = spect_geometry(16, 180.0, 32, 4.0, 32, 4.0)
        return Workload(name, ph, g, 2_000_000, 1, 20, 1e6, 1)
    if name == "torso64":
        ph = torso_phantom(64, 3.2)
        g = spect_geometry(60, 180.0, 64, 3.2, 64, 3.2)
        return Workload(name, ph, g, 100_000_000, 1, 50, 5e6, 2)
    if name == "torso128":
        ph = torso_phantom(128, 2.0, seed=3)
        g = spect_geometry(120, 360.0, 128, 2.0, 128, 2.0)
        return Workload(name, ph, g, 1_000_000_000, 1, 50, 2e7, 3)
    raise KeyError(name)


def serving_mix(n_phantoms: int = 64, seed: int = 5):
    """Mixed-size batch: grids 48/64/96/128 (256 mm field of view), 40-120
    views over 360 deg, heart outer radius 18-28 mm, random defect angle,
    1e6-1e7 counts.  Returns a list of (Phantom, Geometry, counts, seed)."""
    rng = np.random.Generator(np.random.Philox(seed))
    sizes = (48, 64, 96, 128)
    out = []
    for i in range(n_phantoms):
        n = int(sizes[rng.integers(0, len(sizes))])
        h = 256.0 / n
        views = int(rng.integers(40, 121))
        r = float(rng.uniform(18.0, 28.0))
        ph = torso_phantom(n, h, heart_outer=(r, r, 1.2 * r),
                           defect_deg=float(rng.uniform(0.0, 360.0)))
        g = spect_geometry(views, 360.0, n, h, n, h)
        counts = float(10.0 ** rng.uniform(6.0, 7.0))
        out.append((ph, g, counts, 1000 + i))
    return out


def poisson_counts(ybar: np.ndarray, total_counts: float, seed: int) -> np.ndarray:
    """Scale a noiseless projection to ``total_counts`` and draw Poisson
    counts from numpy's Philox generator (seeded)."""
    ybar = np.asarray(ybar, dtype=np.float64)
    s = ybar.sum()
    lam = ybar * (total_counts / s) if s > 0 else ybar
    rng = np.random.Generator(np.random.Philox(seed))
    return rng.poisson(lam).astype(np.float32)


def segments16(phantom: Phantom) -> np.ndarray:
    """Myocardial segment index per voxel (-1 off the heart): 8 azimuthal
    sectors about the heart centre x 2 axial halves."""
    heart = phantom.labels["heart"]
    c = phantom.labels["heart_centre"]
    n = phantom.shape[0]
    x, y, z = _grid(n, phantom.voxel_mm)
    ang = (np.degrees(np.arctan2(y - c[1], x - c[0])) + 360.0) % 360.0
    sector = np.minimum((ang // 45.0).astype(np.int64), 7)
    half = (z >= c[2]).astype(np.int64)
    seg = sector * 2 + half
    return np.where(heart, seg, -1)


def random_events(n_rows: int, n_cols: int, row_len: tuple[int, int], count_max: int, seed: int,
                  rows_used: float = 1.0):
    """Synthetic tally events (row j, column v) of a sparse count matrix, for
    projector and ML-EM tests at chosen row lengths and count ranges.  A
    fraction ``rows_used`` of the rows (chosen at random) holds entries; each
    such row gets a length uniform in ``row_len`` (clipped to n_cols) of
    distinct random columns, each entry a count uniform in 1..count_max
    (repeated events).  Seeded with numpy's Philox generator; returns int32
    rows and cols in random order."""
    rng = np.random.Generator(np.random.Philox(seed))
    used = np.flatnonzero(rng.random(n_rows) < rows_used)
    lens = np.minimum(rng.integers(row_len[0], row_len[1] + 1, len(used)), n_cols)
    rows = np.repeat(used, lens)
    # distinct columns within each row
    cols = np.empty(len(rows), np.int64)
    pos = 0
    for ln in lens:
        cols[pos:pos + ln] = rng.choice(n_cols, ln, replace=False)
        pos += ln
    cnt = rng.integers(1, count_max + 1, len(rows))
    r = np.repeat(rows, cnt).astype(np.int32)
    c = np.repeat(cols, cnt).astype(np.int32)
    order = rng.permutation(len(r))
    return r[order], c[order]


def uniform_events(n_rows: int, n_cols: int, n_events: int, seed: int):
    """Synthetic tally events with row and column independent and uniform
    (repeated pairs add up to counts): a sparse count matrix of any size
    with short rows, e.g. the size class of a 128^3, 120-view system.
    Seeded with numpy's Philox generator; int32 rows and cols."""
    rng = np.random.Generator(np.random.Philox(seed))
    return (rng.integers(0, n_rows, n_events).astype(np.int32),
            rng.integers(0, n_cols, n_events).astype(np.int32))
