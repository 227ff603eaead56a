"""Seeded synthetic inputs for the fictitious-wave FDTD solver.

This module only *builds inputs*: node coordinates, staggered conductivity
arrays and survey geometry.  It holds none of the solver's arithmetic (no
finite-difference weights, no time stepping, no DFT), so both the CUDA path and
the FP64 oracle can consume what it produces without sharing solver code.

Everything here is deterministic: grids are closed-form, random conductivity
perturbations use ``numpy.random.default_rng`` with a fixed seed.

Paper references (Yang, libEMM, arXiv 2304.00233):
  * Sec. 3.7, Eq. 27-29: geometric-progression non-uniform grid and the fixed
    point iteration for its ratio q  -> ``create_nugrid``.
  * Sec. 3.6, Eq. 26: medium homogenisation (arithmetic mean for the
    tangential conductivity, harmonic mean for the normal one)
    -> ``staggered_conductivity``.
  * Sec. 5.6: the solver consumes three resistivity/conductivity cubes of size
    n1*n2*n3, each shifted half a cell along its own axis.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

__all__ = [
    "create_nugrid", "symmetric_axis", "seabed_axis", "uniform_axis",
    "LayeredModel", "Box", "cell_conductivity", "staggered_conductivity",
    "Workload", "whole_space", "marine_1d", "anomaly_3d", "small_case",
    "gradient_survey", "gradient_survey_48", "GRADIENT_SOURCES", "GRADIENT_SOURCES_48",
    "observed_noise", "uneven_grid", "uneven_jobs", "UNEVEN_GRIDS", "WORKLOADS",
]


# ----------------------------------------------------------------------------
# Grid generation (Sec. 3.7)
# ----------------------------------------------------------------------------
def create_nugrid(n: int, length: float, dx: float, tol: float = 1e-15,
                  max_iter: int = 100000) -> np.ndarray:
    """n intervals (n+1 nodes) from 0 to ``length``, first interval ``dx``,
    growing geometrically with ratio q (Eq. 27: L = dx (q^n - 1)/(q - 1)).

    q is found with the fixed-point iteration q <- (L/dx (q-1) + 1)^(1/n)
    of Eq. 28-29, started from q = 1.1, in FP64 with a relative tolerance.
    When n*dx == L the grid is uniform and returned directly.  L < n*dx has no
    solution with q > 1 and raises ValueError.
    """
    if n < 1 or length <= 0 or dx <= 0:
        raise ValueError("create_nugrid: need n>=1, length>0, dx>0")
    if abs(n * dx - length) <= 1e-12 * length:
        return np.arange(n + 1, dtype=np.float64) * dx
    if length < n * dx:
        raise ValueError("create_nugrid: length < n*dx has no stretching q>1")
    q = 1.1
    for _ in range(max_iter):
        qn = (length / dx * (q - 1.0) + 1.0) ** (1.0 / n)
        if abs(qn - q) <= tol * qn:
            q = qn
            break
        q = qn
    else:  # pragma: no cover - the iteration contracts for L > n dx
        raise RuntimeError("create_nugrid: fixed point did not converge")
    i = np.arange(n + 1, dtype=np.float64)
    x = (q ** i - 1.0) * dx / (q - 1.0)
    x[0] = 0.0
    return x


def uniform_axis(n_nodes: int, d: float, centre: float = 0.0) -> np.ndarray:
    """n_nodes equally spaced nodes, symmetric about ``centre``."""
    return centre + (np.arange(n_nodes, dtype=np.float64) - 0.5 * (n_nodes - 1)) * d


def symmetric_axis(n_nodes: int, half_length: float, dx: float) -> np.ndarray:
    """Nodes symmetric about 0, finest spacing ``dx`` at the centre, stretched
    geometrically (``create_nugrid``) towards +-``half_length``.

    Odd n_nodes: a node sits at 0 and each side is create_nugrid((n-1)/2, L, dx).
    Even n_nodes: the two central nodes sit at +-dx/2 and each side is
    dx/2 + create_nugrid(n/2 - 1, L - dx/2, dx).
    """
    if n_nodes % 2:
        side = create_nugrid((n_nodes - 1) // 2, half_length, dx)
        return np.concatenate([-side[:0:-1], side])
    side = 0.5 * dx + create_nugrid(n_nodes // 2 - 1, half_length - 0.5 * dx, dx)
    return np.concatenate([-side[::-1], side])


def seabed_axis(z_seabed: float, n_up: int, len_up: float, n_down: int,
                len_down: float, dz: float) -> np.ndarray:
    """z (positive down) stretched away from the seabed in both directions:
    ``n_up`` intervals covering ``len_up`` above it, ``n_down`` intervals
    covering ``len_down`` below it, both starting with spacing ``dz``.
    Returns n_up + n_down + 1 nodes."""
    up = create_nugrid(n_up, len_up, dz)
    down = create_nugrid(n_down, len_down, dz)
    return np.concatenate([z_seabed - up[:0:-1], z_seabed + down])


# ----------------------------------------------------------------------------
# Conductivity models and homogenisation (Sec. 3.6)
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Box:
    """Axis-aligned isotropic anomaly."""
    lo: Sequence[float]
    hi: Sequence[float]
    sigma: float


@dataclasses.dataclass
class LayeredModel:
    """1-D VTI layering in z (positive down) plus optional isotropic boxes.

    ``tops`` are layer top depths (ascending, the first one is -inf implied),
    ``sigma_h``/``sigma_v`` the layer conductivities (S/m)."""
    tops: Sequence[float]
    sigma_h: Sequence[float]
    sigma_v: Sequence[float]
    boxes: Sequence[Box] = ()

    def breakpoints(self) -> List[float]:
        pts = list(self.tops[1:])
        for b in self.boxes:
            pts += [b.lo[2], b.hi[2]]
        return sorted(set(pts))

    def layer_at(self, z: float) -> int:
        k = 0
        for i, t in enumerate(self.tops):
            if z >= t:
                k = i
        return k


def _overlap(a0: np.ndarray, a1: np.ndarray, b0: float, b1: float) -> np.ndarray:
    return np.clip(np.minimum(a1, b1) - np.maximum(a0, b0), 0.0, None) / (a1 - a0)


def cell_conductivity(model: LayeredModel, x: np.ndarray, y: np.ndarray,
                      z: np.ndarray):
    """Cell-centred (sigma_h, sigma_v), shape [n3-1][n2-1][n1-1].

    Inside each cell the z-range is cut at every layer/box boundary.  On each
    z piece the conductivity is averaged arithmetically over the cell's x-y
    face (box volume fraction).  sigma_h is the arithmetic mean of the pieces
    over z, sigma_v the harmonic mean over z (Eq. 26: tangential = resistors in
    parallel, normal = resistors in series)."""
    nx, ny, nz = len(x) - 1, len(y) - 1, len(z) - 1
    sh = np.empty((nz, ny, nx))
    sv = np.empty((nz, ny, nx))
    bps = model.breakpoints()
    box_fx = [_overlap(x[:-1], x[1:], b.lo[0], b.hi[0]) for b in model.boxes]
    box_fy = [_overlap(y[:-1], y[1:], b.lo[1], b.hi[1]) for b in model.boxes]
    for k in range(nz):
        z0, z1 = z[k], z[k + 1]
        cuts = [z0] + [p for p in bps if z0 < p < z1] + [z1]
        acc_h = np.zeros((ny, nx))
        acc_r = np.zeros((ny, nx))
        for a, b in zip(cuts[:-1], cuts[1:]):
            zm = 0.5 * (a + b)
            lay = model.layer_at(zm)
            bh = np.full((ny, nx), float(model.sigma_h[lay]))
            bv = np.full((ny, nx), float(model.sigma_v[lay]))
            for bx, fx, fy in zip(model.boxes, box_fx, box_fy):
                if bx.lo[2] <= zm < bx.hi[2]:
                    f = fy[:, None] * fx[None, :]
                    bh = (1 - f) * bh + f * bx.sigma
                    bv = (1 - f) * bv + f * bx.sigma
            acc_h += (b - a) * bh
            acc_r += (b - a) / bv
        sh[k] = acc_h / (z1 - z0)
        sv[k] = (z1 - z0) / acc_r
    return sh, sv


def staggered_conductivity(sh: np.ndarray, sv: np.ndarray, x: np.ndarray,
                           y: np.ndarray, z: np.ndarray) -> np.ndarray:
    """Staggered (sigma_xx, sigma_yy, sigma_zz) at the E_x, E_y, E_z sample
    positions, shape [3][n3][n2][n1], from cell values.

    E_x sits at (x_{i+1/2}, y_j, z_k): the edge is shared by the (up to) four
    cells adjacent in y and z; sigma_xx is their area-weighted arithmetic mean
    of sigma_h.  Same for E_y; E_z averages sigma_v over the four cells adjacent
    in x and y.  Indices past the last cell clamp to it (half node beyond the
    last interior node, and the domain edges)."""
    n1, n2, n3 = len(x), len(y), len(z)
    dx, dy, dz = np.diff(x), np.diff(y), np.diff(z)

    def pair(n_nodes, d):
        # for node j: neighbouring cells j-1 and j (clamped) and their widths
        j = np.arange(n_nodes)
        lo = np.clip(j - 1, 0, n_nodes - 2)
        hi = np.clip(j, 0, n_nodes - 2)
        return lo, hi, d[lo], d[hi]

    def own(n_nodes):
        return np.clip(np.arange(n_nodes), 0, n_nodes - 2)

    out = np.empty((3, n3, n2, n1))
    # sigma_xx: cells (own x, pair y, pair z)
    ix = own(n1)
    ylo, yhi, wylo, wyhi = pair(n2, dy)
    zlo, zhi, wzlo, wzhi = pair(n3, dz)
    s = 0.0
    w = 0.0
    for zc, wz in ((zlo, wzlo), (zhi, wzhi)):
        for yc, wy in ((ylo, wylo), (yhi, wyhi)):
            ww = wz[:, None, None] * wy[None, :, None]
            s = s + ww * sh[zc][:, yc][:, :, ix]
            w = w + ww
    out[0] = s / w
    # sigma_yy: cells (pair x, own y, pair z)
    iy = own(n2)
    xlo, xhi, wxlo, wxhi = pair(n1, dx)
    s = 0.0
    w = 0.0
    for zc, wz in ((zlo, wzlo), (zhi, wzhi)):
        for xc, wx in ((xlo, wxlo), (xhi, wxhi)):
            ww = wz[:, None, None] * wx[None, None, :]
            s = s + ww * sh[zc][:, iy][:, :, xc]
            w = w + ww
    out[1] = s / w
    # sigma_zz: cells (pair x, pair y, own z), vertical conductivity
    iz = own(n3)
    s = 0.0
    w = 0.0
    for yc, wy in ((ylo, wylo), (yhi, wyhi)):
        for xc, wx in ((xlo, wxlo), (xhi, wxhi)):
            ww = wy[None, :, None] * wx[None, None, :]
            s = s + ww * sv[iz][:, yc][:, :, xc]
            w = w + ww
    out[2] = s / w
    return out


# ----------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    """Everything a forward solve needs, as plain arrays.

    ``sigma`` is the staggered conductivity [3][n3][n2][n1], already rounded to
    FP32 (and stored as FP64) so that the FP32 device path and the FP64 oracle
    see bit-identical medium values."""
    name: str
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    sigma: np.ndarray
    rd: int
    nb: int
    ne: int
    src: np.ndarray            # [3]
    src_az: float
    src_dip: float
    moment: float
    rec: np.ndarray            # [nrec][3]
    freqs: np.ndarray          # Hz
    omega0: float
    fmax: float
    t_max: float               # fictitious time simulated
    volume: bool = False
    nt: Optional[int] = None   # fixed step count (else ceil(t_max/dt))
    sigma_h: Optional[np.ndarray] = None   # cell values [n3-1][n2-1][n1-1] behind sigma, when kept
    sigma_v: Optional[np.ndarray] = None

    @property
    def shape(self):
        return (len(self.x), len(self.y), len(self.z))

    @property
    def npad(self):
        p = 2 * (self.nb + self.ne)
        return (len(self.x) + p, len(self.y) + p, len(self.z) + p)

    @property
    def padded_cells(self) -> int:
        a, b, c = self.npad
        return a * b * c


def _f32(a: np.ndarray) -> np.ndarray:
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def whole_space(n: int = 64, d: float = 50.0, rd: int = 2) -> Workload:
    """Homogeneous whole space, sigma = 1 S/m, uniform n^3 nodes at spacing d,
    x-directed unit dipole at the origin, one frequency 0.5 Hz, 32 inline
    receivers at offsets 200..1800 m."""
    x = uniform_axis(n, d)
    sig = np.ones((3, n, n, n))
    rec = np.zeros((32, 3))
    rec[:, 0] = np.linspace(200.0, 1800.0, 32)
    return Workload("whole_space_64", x, x.copy(), x.copy(), _f32(sig), rd, 10,
                    rd + 5, np.zeros(3), 0.0, 0.0, 1.0, rec,
                    np.array([0.5]), 2 * math.pi, 1.0, 3.7)


def _marine_model(with_resistor: bool = True) -> LayeredModel:
    tops = [-1e30, 1000.0]
    sh = [3.3, 1.0]
    sv = [3.3, 0.5]
    if with_resistor:
        tops += [2000.0, 2100.0]
        sh += [0.02, 1.0]
        sv += [0.02, 0.5]
    return LayeredModel(tops, sh, sv)


def marine_1d(nxy: int = 128, nz: int = 96, rd: int = 2) -> Workload:
    """Layered marine VTI model: 1000 m of sea water (3.3 S/m), sediment
    (sigma_h = 1, sigma_v = 0.5 S/m) with a 100 m resistor (0.02 S/m) whose top
    is 1000 m below the seabed.  NU grid 128 x 128 x 96 nodes, 40 m cells at the
    centre and at the seabed stretched to ~200 m.  Source 50 m above the seabed,
    64 seabed receivers, frequencies 0.25/0.75/1.25 Hz."""
    x = symmetric_axis(nxy, 6400.0, 40.0)
    n_up = 16
    z = seabed_axis(1000.0, n_up, 1000.0, nz - n_up - 1, 8000.0, 40.0)
    model = _marine_model(True)
    sh, sv = cell_conductivity(model, x, x, z)
    sig = staggered_conductivity(sh, sv, x, x, z)
    rec = np.zeros((64, 3))
    rec[:, 0] = -6300.0 + 200.0 * np.arange(64)
    rec[:, 2] = 1000.0
    return Workload("marine_1d_128x128x96", x, x.copy(), z, _f32(sig), rd, 10,
                    rd + 5, np.array([0.0, 0.0, 950.0]), 0.0, 0.0, 1.0, rec,
                    np.array([0.25, 0.75, 1.25]), 2 * math.pi, 1.0, 6.4)


def marine_1d_air(nxy: int = 128, nz: int = 96, rd: int = 2) -> Workload:
    """The layered marine model of ``marine_1d`` with the sea surface (z = 0)
    as an interface with air, on a grid uniform in x and y (100 m, as the
    DFT of the air boundary needs) and the same stretched z axis; same
    source, receivers and frequencies."""
    x = (np.arange(nxy) - 0.5 * (nxy - 1)) * 100.0
    n_up = 16
    z = seabed_axis(1000.0, n_up, 1000.0, nz - n_up - 1, 8000.0, 40.0)
    model = _marine_model(True)
    sh, sv = cell_conductivity(model, x, x, z)
    sig = staggered_conductivity(sh, sv, x, x, z)
    rec = np.zeros((64, 3))
    rec[:, 0] = -6300.0 + 200.0 * np.arange(64)
    rec[:, 2] = 1000.0
    return Workload("marine_1d_air_128x128x96", x, x.copy(), z, _f32(sig), rd, 10,
                    rd + 5, np.array([0.0, 0.0, 950.0]), 0.0, 0.0, 1.0, rec,
                    np.array([0.25, 0.75, 1.25]), 2 * math.pi, 1.0, 6.4)


def anomaly_3d(seed: int = 230400233) -> Workload:
    """Marine background of ``marine_1d`` on a 256 x 256 x 160 NU grid, plus a
    4 x 3 km x 100 m resistive block (0.01 S/m) at 2000-2100 m depth and a
    lognormal multiplier exp(0.3 g), g ~ N(0,1) i.i.d. per sediment cell.
    8th order (rd=4), 201 receivers on three seabed lines, volume DFT on."""
    x = symmetric_axis(256, 12750.0, 40.0)
    z = seabed_axis(1000.0, 16, 1000.0, 143, 14300.0, 40.0)
    model = _marine_model(True)
    model.boxes = [Box((-2000.0, -1500.0, 2000.0), (2000.0, 1500.0, 2100.0), 0.01)]
    sh, sv = cell_conductivity(model, x, x, z)
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(sh.shape)
    zc = 0.5 * (z[:-1] + z[1:])
    mult = np.where((zc > 1000.0)[:, None, None], np.exp(0.3 * g), 1.0)
    sh = sh * mult
    sv = sv * mult
    sig = staggered_conductivity(sh, sv, x, x, z)
    xs = -6600.0 + 200.0 * np.arange(67)
    rec = np.array([[xr, yr, 1000.0] for yr in (-1000.0, 0.0, 1000.0) for xr in xs])
    return Workload("anomaly_3d_256x256x160", x, x.copy(), z, _f32(sig), 4, 10, 9,
                    np.array([0.0, 0.0, 950.0]), 0.0, 0.0, 1.0, rec,
                    np.array([0.25, 0.75, 1.25]), 2 * math.pi, 1.0, 6.46,
                    volume=True)


# transmitters of the gradient survey: a tow line 50 m above the seabed
GRADIENT_SOURCES = np.array([[-2800.0 + 800.0 * k, 0.0, 950.0] for k in range(8)])


def gradient_survey(with_resistor: bool = False, nt: Optional[int] = None) -> Workload:
    """Least-squares gradient survey: the marine layering of ``marine_1d`` on a
    192 x 192 x 128 NU grid (x, y 96 cells per side over 9550 m from 40 m; z
    16 cells over 1000 m above the seabed and 111 over 11150 m below it, from
    40 m), the receivers of ``marine_1d``, the transmitter at the first of
    ``GRADIENT_SOURCES``.  The observed data come from the model with the
    resistor; the gradient is taken at the model without it.  The cell
    values sigma_h, sigma_v are kept (the gradient is with respect to them)."""
    x = symmetric_axis(192, 9550.0, 40.0)
    z = seabed_axis(1000.0, 16, 1000.0, 111, 11150.0, 40.0)
    sh, sv = cell_conductivity(_marine_model(with_resistor), x, x, z)
    sig = staggered_conductivity(sh, sv, x, x, z)
    rec = np.zeros((64, 3))
    rec[:, 0] = -6300.0 + 200.0 * np.arange(64)
    rec[:, 2] = 1000.0
    name = "gradient_survey_192x192x128" + ("_resistor" if with_resistor else "")
    return Workload(name, x, x.copy(), z, _f32(sig), 2, 10, 7, GRADIENT_SOURCES[0].copy(), 0.0, 0.0, 1.0,
                    rec, np.array([0.25, 0.75, 1.25]), 2 * math.pi, 1.0, 6.4, nt=nt, sigma_h=sh, sigma_v=sv)


# transmitters of the small copy of the gradient survey
GRADIENT_SOURCES_48 = np.array([[-400.0, 0.0, 950.0], [400.0, 0.0, 950.0]])


def gradient_survey_48(with_resistor: bool = False, nt: int = 200) -> Workload:
    """The gradient survey on a 48 x 48 x 48 copy small enough for the FP64
    oracle: x, y 24 cells per side over 2400 m from 40 m; z 16 cells over
    1000 m above the seabed and 31 over 3200 m below it; receivers every
    200 m from -2100 to 2100 m on the seabed; transmitters at
    ``GRADIENT_SOURCES_48``; a fixed, short step count."""
    x = symmetric_axis(48, 2400.0, 40.0)
    z = seabed_axis(1000.0, 16, 1000.0, 31, 3200.0, 40.0)
    sh, sv = cell_conductivity(_marine_model(with_resistor), x, x, z)
    sig = staggered_conductivity(sh, sv, x, x, z)
    rec = np.zeros((22, 3))
    rec[:, 0] = -2100.0 + 200.0 * np.arange(22)
    rec[:, 2] = 1000.0
    name = "gradient_survey_48" + ("_resistor" if with_resistor else "")
    return Workload(name, x, x.copy(), z, _f32(sig), 2, 10, 7, GRADIENT_SOURCES_48[0].copy(), 0.0, 0.0, 1.0,
                    rec, np.array([0.25, 0.75, 1.25]), 2 * math.pi, 1.0, 6.4, nt=nt, sigma_h=sh, sigma_v=sv)


def _stretched_length(n: int, d0: float = 40.0, d1: float = 200.0) -> float:
    # length of n geometric cells growing from d0 to d1 (ratio (d1/d0)^(1/(n-1)))
    q = (d1 / d0) ** (1.0 / (n - 1))
    return d0 * (q ** n - 1.0) / (q - 1.0)


def uneven_grid(n1: int, n3: int) -> Workload:
    """One problem of the uneven-grid work list: the layered marine model
    (with the resistor) on n1 x n1 x n3 nodes, x and y n1/2 cells per side
    and z 16 cells above the seabed over 1000 m and n3 - 17 below it, every
    axis growing from 40 m to about 200 m; the transmitter 50 m above the
    seabed at the grid centre, seabed receivers every 200 m from -3100 m to
    3100 m (those within 80 % of the half-width on smaller grids)."""
    half = n1 // 2
    L = _stretched_length(half)
    x = symmetric_axis(n1, L, 40.0)
    n_down = n3 - 17
    z = seabed_axis(1000.0, 16, 1000.0, n_down, _stretched_length(n_down), 40.0)
    sh, sv = cell_conductivity(_marine_model(True), x, x, z)
    sig = staggered_conductivity(sh, sv, x, x, z)
    xr = -3100.0 + 200.0 * np.arange(32)
    xr = xr[np.abs(xr) <= 0.8 * L]
    rec = np.zeros((len(xr), 3))
    rec[:, 0] = xr
    rec[:, 2] = 1000.0
    return Workload(f"uneven_{n1}x{n1}x{n3}", x, x.copy(), z, _f32(sig), 2, 10, 7, np.array([0.0, 0.0, 950.0]),
                    0.0, 0.0, 1.0, rec, np.array([0.25, 0.75, 1.25]), 2 * math.pi, 1.0, 6.4)


# the uneven-grid work list: 3 x 96^3, 3 x 160 x 160 x 120, 2 x 200 x 200 x 140 nodes
UNEVEN_GRIDS = [(96, 96)] * 3 + [(160, 120)] * 3 + [(200, 140)] * 2


def uneven_jobs() -> List[Workload]:
    """The eight problems of the uneven-grid work list (``UNEVEN_GRIDS``)."""
    return [uneven_grid(a, b) for a, b in UNEVEN_GRIDS]


def observed_noise(shape, seed: int = 230400234, level: float = 0.02) -> np.ndarray:
    """Multiplicative complex noise 1 + level (g1 + i g2) / sqrt(2), g ~ N(0, 1)
    i.i.d., for synthetic observed data d = G (1 + noise)."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(tuple(shape) + (2,))
    return 1.0 + level * (g[..., 0] + 1j * g[..., 1]) / math.sqrt(2.0)


def small_case(n=(40, 36, 30), rd: int = 2, seed: int = 7, nt: int = 120,
               volume: bool = True, nb: int = 6, nfreq: int = 2) -> Workload:
    """Small NU VTI case for element-wise parity tests: random smooth
    stretching per axis, random positive conductivity (log-uniform 0.3..3 S/m)
    per staggered sample, a tilted dipole and a handful of receivers."""
    rng = np.random.default_rng(seed)

    def axis(m, d0):
        # spacing grows/shrinks smoothly: d_i = d0 * exp(0.25 sin(...))
        t = np.linspace(0, 1, m - 1)
        d = d0 * np.exp(0.3 * np.sin(2 * math.pi * (t + rng.uniform())))
        return np.concatenate([[0.0], np.cumsum(d)]) - 0.5 * d.sum()

    x, y, z = axis(n[0], 50.0), axis(n[1], 45.0), axis(n[2], 40.0)
    sig = np.exp(rng.uniform(math.log(0.3), math.log(3.0), (3, n[2], n[1], n[0])))
    c = np.array([0.5 * (x[0] + x[-1]), 0.5 * (y[0] + y[-1]), 0.5 * (z[0] + z[-1])])
    src = c + np.array([13.0, -7.0, 5.0])
    span = np.array([x[-1] - x[0], y[-1] - y[0], z[-1] - z[0]])
    rec = c + (rng.uniform(-0.3, 0.3, (7, 3)) * span)
    freqs = np.array([0.5, 1.5, 2.5, 3.5])[:nfreq]
    return Workload(f"small_{n[0]}x{n[1]}x{n[2]}_rd{rd}", x, y, z, _f32(sig), rd,
                    nb, rd + 3, src, 0.4, 0.3, 1.0, rec, freqs, 2 * math.pi,
                    2.0, 0.0, volume=volume, nt=nt)


WORKLOADS = {
    "whole_space_64": whole_space,
    "marine_1d_128x128x96": marine_1d,
    "anomaly_3d_256x256x160": anomaly_3d,
}
