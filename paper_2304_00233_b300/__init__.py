"""B300-native fictitious-wave FDTD (libEMM's method, Yang, arXiv 2304.00233).

Thin Python binding of the C ABI in ``include/emm.h`` (``libemm.so``): the
functions below only marshal arguments through ctypes.  Every step of the time
loop runs in the library's CUDA kernels; PyTorch provides device memory and
streams.  There is no CPU fallback: if ``libemm.so`` is missing or cannot be
loaded, every call raises.

    grid = make_grid(x, y, z, rd=2, nb=10, ne=7)
    survey = Survey(omega0=2*pi, fmax=1.0, sigma_min=0.02, nt=7000,
                    src=(0, 0, 950), rec=rec_xyz, freqs=[0.25, 0.75, 1.25])
    G, vol = forward(grid, survey, sigma)     # sigma: [3][n3][n2][n1] float32

``G`` is complex128 [nrec][6][nfreq]: G^EE (components 0..2) and G^HE (3..5)
of Eq. 7; ``vol`` is [6][nfreq][n3][n2][n1] when ``survey.volume``.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import math
import os
from typing import Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBRARY_PATH = os.path.join(_HERE, "libemm.so")

(EMM_OK, EMM_EINVAL, EMM_ENOMEM, EMM_EOUTSIDE, EMM_ECFL, EMM_ECUDA, EMM_EWORKSPACE, EMM_EDEVICE,
 EMM_ETIMEOUT) = range(9)
# EMM_VOLUME_RING: leapfrog steps one volume-DTFT launch covers (the field
# ring of a one-transmitter solve with the volume DTFT)
VOLUME_RING = 8
JOBS_LIST, JOBS_SEQUENTIAL, JOBS_STREAMS = range(3)
JOBS_STRATEGIES = ("list", "sequential", "streams")
TAB_NODES, TAB_HALF, TAB_DPLUS, TAB_DMINUS, TAB_SLAB_INT, TAB_SLAB_HALF = range(6)
COMPONENTS = ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz")
EXPORTED = ("emm_make_grid", "emm_free_grid", "emm_grid_query", "emm_grid_tables",
            "emm_time_step", "emm_cpml_tables", "emm_locate", "emm_workspace_size",
            "emm_forward", "emm_forward_timed", "emm_status", "emm_strerror",
            "emm_forward_static", "emm_gradient_workspace_size", "emm_gradient",
            "emm_batch_workspace_size", "emm_forward_batch", "emm_forward_converge",
            "emm_gradient_stored_workspace_size", "emm_gradient_stored", "emm_misfit_gradient",
            "emm_stagger_workspace_size", "emm_stagger_sigma", "emm_stagger_sigma_adjoint",
            "emm_jobs_workspace_size", "emm_forward_jobs", "emm_jobs_tune", "emm_plan_create", "emm_plan_run",
            "emm_plan_destroy", "emm_persist_workspace_size", "emm_forward_persistent", "emm_persist_tune",
            "emm_persist_plan_create", "emm_persist_plan_run", "emm_persist_plan_destroy",
            "emm_wave_workspace_size", "emm_forward_wave")


class EmmError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} (code {code})")


_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)


class _GridDesc(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("x", _D * 3), ("rd", C.c_int), ("nb", C.c_int), ("ne", C.c_int)]


class _GridInfo(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("npad", C.c_int * 3), ("rd", C.c_int), ("nb", C.c_int),
                ("ne", C.c_int), ("cells", C.c_size_t)]


class _Timing(C.Structure):
    _fields_ = [("every", C.c_int), ("samples", C.c_int), ("e_ms", C.c_double),
                ("h_ms", C.c_double), ("total_ms", C.c_double), ("loop_ms", C.c_double),
                ("v_ms", C.c_double)]


class _Survey(C.Structure):
    _fields_ = [("omega0", C.c_double), ("fmax", C.c_double), ("sigma_min", C.c_double),
                ("dt", C.c_double), ("nt", C.c_int), ("src", C.c_double * 3),
                ("src_az", C.c_double), ("src_dip", C.c_double), ("moment", C.c_double),
                ("nrec", C.c_int), ("rec", _D), ("nfreq", C.c_int), ("freqs", _D),
                ("volume", C.c_int), ("src_kind", C.c_int),
                ("src_length", C.c_double), ("src_points", C.c_int), ("airwave", C.c_int),
                ("tile_shape", C.c_int)]


class _Job(C.Structure):
    _fields_ = [("grid", C.c_void_p), ("survey", C.POINTER(_Survey)), ("sigma", C.c_void_p),
                ("rec_out", C.c_void_p)]


class _Task(C.Structure):
    _fields_ = [("grid", C.c_void_p), ("survey", C.POINTER(_Survey)), ("sigma", C.c_void_p),
                ("nsrc", C.c_int), ("src_pos", _D), ("rec_out", C.c_void_p)]


class PersistOpts(C.Structure):
    """``emm_persist_opts``: resident CTAs per SM (0: as many as fit), a cap
    on all CTAs (0: none), the bound of one grid-barrier wait in seconds
    (<= 0: 1 s), for tests only a CTA that withholds its first arrival
    (-1: none), and the tile shape (0: 32 x 8 x 2 cells, 1: 32 x 4 x 4)."""
    _fields_ = [("ctas_per_sm", C.c_int), ("max_ctas", C.c_int), ("wait_s", C.c_double),
                ("skip_arrival", C.c_int), ("tile_shape", C.c_int)]

    def __init__(self, ctas_per_sm=0, max_ctas=0, wait_s=0.0, skip_arrival=-1, tile_shape=0):
        super().__init__(int(ctas_per_sm), int(max_ctas), float(wait_s), int(skip_arrival), int(tile_shape))

    def key(self):
        """(tile shape, resident CTAs per SM) of these options."""
        return (int(self.tile_shape), int(self.ctas_per_sm))

    def __repr__(self):
        return (f"PersistOpts(ctas_per_sm={self.ctas_per_sm}, max_ctas={self.max_ctas}, wait_s={self.wait_s}, "
                f"skip_arrival={self.skip_arrival}, tile_shape={self.tile_shape})")


_lib = None


def load_library(path: str = LIBRARY_PATH) -> C.CDLL:
    """Load libemm.so (built by ``python -m paper_2304_00233_b300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libemm.so not found at {path}: build it with "
                           "`python -m paper_2304_00233_b300.build` (no CPU fallback exists)")
    lib = C.CDLL(path)
    V = C.c_void_p
    sig = {
        "emm_make_grid": ([C.POINTER(_GridDesc), C.POINTER(V)], C.c_int),
        "emm_free_grid": ([V], None),
        "emm_grid_query": ([V, C.POINTER(_GridInfo)], C.c_int),
        "emm_grid_tables": ([V, C.c_int, C.c_int, _D, _I], C.c_int),
        "emm_time_step": ([V, C.c_double, C.c_double, _D, _D, _D], C.c_int),
        "emm_cpml_tables": ([V, C.c_int, C.c_double, C.c_double, C.c_double, _D], C.c_int),
        "emm_locate": ([V, C.c_int, _D, _I, _D], C.c_int),
        "emm_workspace_size": ([V, C.POINTER(_Survey), C.POINTER(C.c_size_t)], C.c_int),
        "emm_forward": ([V, C.POINTER(_Survey), V, V, C.c_size_t, V, V, V], C.c_int),
        "emm_forward_timed": ([V, C.POINTER(_Survey), V, V, C.c_size_t, V, V, V,
                               C.POINTER(_Timing)], C.c_int),
        "emm_status": ([V, _I, V], C.c_int),
        "emm_forward_static": ([V, C.POINTER(_Survey), V, V, V, V, _I], C.c_int),
        "emm_batch_workspace_size": ([V, C.POINTER(_Survey), C.c_int, C.POINTER(C.c_size_t)], C.c_int),
        "emm_forward_batch": ([V, C.POINTER(_Survey), C.c_int, _D, V, V, C.c_size_t, V, V], C.c_int),
        "emm_forward_converge": ([V, C.POINTER(_Survey), V, V, C.c_size_t, V, V, V, _I], C.c_int),
        "emm_gradient_workspace_size": ([V, C.POINTER(_Survey), C.c_int, C.POINTER(C.c_size_t)], C.c_int),
        "emm_gradient": ([V, C.POINTER(_Survey), V, V, C.c_int, V, C.c_size_t, V, V, V], C.c_int),
        "emm_gradient_stored_workspace_size": ([V, C.POINTER(_Survey), C.c_int, C.c_int, C.POINTER(C.c_size_t)],
                                               C.c_int),
        "emm_gradient_stored": ([V, C.POINTER(_Survey), V, V, C.c_int, C.c_int, V, C.c_size_t, V, V, V], C.c_int),
        "emm_misfit_gradient": ([V, C.POINTER(_Survey), V, V, V, C.c_int, C.c_int, V, C.c_size_t, V, V, V, V],
                                C.c_int),
        "emm_stagger_workspace_size": ([V, C.POINTER(C.c_size_t)], C.c_int),
        "emm_stagger_sigma": ([V, V, V, V, C.c_size_t, V, V], C.c_int),
        "emm_stagger_sigma_adjoint": ([V, V, V, C.c_size_t, V, V, V], C.c_int),
        "emm_jobs_workspace_size": ([C.c_int, C.POINTER(_Job), C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)],
                                    C.c_int),
        "emm_forward_jobs": ([C.c_int, C.POINTER(_Job), C.c_int, V, C.c_size_t, V], C.c_int),
        "emm_jobs_tune": ([C.c_int, C.POINTER(_Job), V, C.c_size_t, C.c_int, V, _D, _I], C.c_int),
        "emm_persist_workspace_size": ([C.c_int, C.POINTER(_Task), C.POINTER(C.c_size_t),
                                        C.POINTER(C.c_size_t)], C.c_int),
        "emm_forward_persistent": ([C.c_int, C.POINTER(_Task), C.POINTER(PersistOpts), V, C.c_size_t, V], C.c_int),
        "emm_persist_tune": ([C.c_int, C.POINTER(_Task), V, C.c_size_t, C.c_int, V, _I, C.POINTER(PersistOpts), _D,
                              C.POINTER(PersistOpts)], C.c_int),
        "emm_persist_plan_create": ([C.c_int, C.POINTER(_Task), C.POINTER(PersistOpts), V, C.c_size_t, V,
                                     C.POINTER(V)], C.c_int),
        "emm_persist_plan_run": ([V, V], C.c_int),
        "emm_persist_plan_destroy": ([V], None),
        "emm_wave_workspace_size": ([V, C.POINTER(_Survey), C.c_int, C.POINTER(C.c_size_t)], C.c_int),
        "emm_forward_wave": ([V, C.POINTER(_Survey), V, C.c_int, V, C.c_size_t, V, V], C.c_int),
        "emm_plan_create": ([V, C.POINTER(_Survey), V, V, C.c_size_t, V, V, V, C.POINTER(V)], C.c_int),
        "emm_plan_run": ([V, V, V], C.c_int),
        "emm_plan_destroy": ([V], None),
        "emm_strerror": ([C.c_int], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def strerror(code: int) -> str:
    return load_library().emm_strerror(int(code)).decode()


def _check(code: int, what: str):
    if code != EMM_OK:
        raise EmmError(code, what)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _dp(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(_D)


class Grid:
    """Handle of an ``emm_grid`` (padded nodes, half nodes, FD rows)."""

    def __init__(self, x, y, z, rd: int = 2, nb: int = 10, ne: Optional[int] = None):
        lib = load_library()
        self._axes = [_f64(x), _f64(y), _f64(z)]
        self.rd, self.nb = int(rd), int(nb)
        self.ne = int(rd + 5 if ne is None else ne)
        d = _GridDesc()
        d.n = (C.c_int * 3)(*[len(a) for a in self._axes])
        d.x = (_D * 3)(*[_dp(a) for a in self._axes])
        d.rd, d.nb, d.ne = self.rd, self.nb, self.ne
        h = C.c_void_p()
        _check(lib.emm_make_grid(C.byref(d), C.byref(h)), "emm_make_grid")
        self._h = h
        info = _GridInfo()
        _check(lib.emm_grid_query(h, C.byref(info)), "emm_grid_query")
        self.n = tuple(info.n)
        self.npad = tuple(info.npad)
        self.cells = int(info.cells)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.emm_free_grid(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def table(self, axis: int, kind: int):
        """Test hook: ``emm_grid_tables`` as numpy arrays (coef, idx)."""
        np_ = self.npad[axis]
        m = 2 * self.rd
        coef = idx = None
        if kind == TAB_NODES:
            coef = np.zeros(np_ + 1)
        elif kind == TAB_HALF:
            coef = np.zeros(np_)
        elif kind in (TAB_DPLUS, TAB_DMINUS):
            coef, idx = np.zeros((np_, m)), np.zeros(np_, np.int32)
        else:
            idx = np.zeros(np_, np.int32)
        _check(load_library().emm_grid_tables(self._h, axis, kind, _dp(coef),
                                              None if idx is None else idx.ctypes.data_as(_I)),
               "emm_grid_tables")
        return coef, idx

    def time_step(self, sigma_min: float, omega0: float) -> Tuple[float, float, float]:
        """(dt, eta, vmax) of Sec. 3.2."""
        dt, eta, vmax = C.c_double(), C.c_double(), C.c_double()
        _check(load_library().emm_time_step(self._h, sigma_min, omega0, C.byref(dt), C.byref(eta),
                                            C.byref(vmax)), "emm_time_step")
        return dt.value, eta.value, vmax.value

    def cpml_tables(self, axis: int, vmax: float, fmax: float, dt: float) -> np.ndarray:
        ab = np.zeros((4, 2 * self.nb))
        _check(load_library().emm_cpml_tables(self._h, axis, vmax, fmax, dt, _dp(ab)), "emm_cpml_tables")
        return ab

    def locate(self, comp: int, pos) -> Tuple[np.ndarray, np.ndarray]:
        pos = _f64(pos)
        start = np.zeros(3, np.int32)
        w = np.zeros((3, 2 * self.rd))
        _check(load_library().emm_locate(self._h, comp, _dp(pos), start.ctypes.data_as(_I), _dp(w)),
               "emm_locate")
        return start, w


def make_grid(x, y, z, rd: int = 2, nb: int = 10, ne: Optional[int] = None) -> Grid:
    return Grid(x, y, z, rd, nb, ne)


@dataclasses.dataclass
class Survey:
    """One transmitter, its receivers and the frequencies (``emm_survey``)."""
    omega0: float
    fmax: float
    sigma_min: float
    nt: int
    src: Sequence[float] = (0.0, 0.0, 0.0)
    rec: Optional[np.ndarray] = None
    freqs: Sequence[float] = (1.0,)
    dt: float = 0.0
    src_az: float = 0.0
    src_dip: float = 0.0
    moment: float = 1.0
    volume: bool = False
    src_kind: int = 0          # 0: electric dipole J; 1: magnetic dipole M
    src_length: float = 0.0    # > 0: an antenna of this length (m), as src_points sub-dipoles
    src_points: int = 1
    airwave: bool = False      # air above the top interior node (needs uniform x, y)
    tile_shape: int = 0        # stencil tile: 0 = 32 x 8 x 2 cells, 1 = 32 x 4 x 4

    def _c(self) -> Tuple[_Survey, list]:
        rec = _f64(np.zeros((0, 3)) if self.rec is None else self.rec).reshape(-1, 3)
        freqs = _f64(self.freqs)
        s = _Survey()
        s.omega0, s.fmax, s.sigma_min, s.dt = self.omega0, self.fmax, self.sigma_min, self.dt
        s.nt = int(self.nt)
        s.src = (C.c_double * 3)(*[float(v) for v in self.src])
        s.src_az, s.src_dip, s.moment = self.src_az, self.src_dip, self.moment
        s.nrec = rec.shape[0]
        s.rec = _dp(rec) if rec.shape[0] else None
        s.nfreq = len(freqs)
        s.freqs = _dp(freqs) if len(freqs) else None
        s.volume = int(bool(self.volume))
        s.src_kind = int(self.src_kind)
        s.src_length, s.src_points = float(self.src_length), int(self.src_points)
        s.airwave = int(bool(self.airwave))
        s.tile_shape = int(self.tile_shape)
        return s, [rec, freqs]   # the arrays must outlive every use of the struct

    @property
    def nrec(self) -> int:
        return 0 if self.rec is None else int(np.asarray(self.rec).reshape(-1, 3).shape[0])


def workspace_size(grid: Grid, survey: Survey) -> int:
    s, keep = survey._c()
    out = C.c_size_t()
    _check(load_library().emm_workspace_size(grid.handle, C.byref(s), C.byref(out)), "emm_workspace_size")
    return int(out.value)


class Workspace:
    """Device buffers of one forward configuration, reusable across calls."""

    def __init__(self, grid: Grid, survey: Survey, device=None):
        import torch
        self.device = torch.device("cuda" if device is None else device)
        self.bytes = workspace_size(grid, survey)
        self.ws = torch.empty(self.bytes + 256, dtype=torch.uint8, device=self.device)
        off = (-self.ws.data_ptr()) % 256
        self.ptr = self.ws.data_ptr() + off
        nf = len(survey.freqs)
        self.rec = torch.zeros((max(survey.nrec, 1), 6, nf, 2), dtype=torch.float64, device=self.device)
        self.vol = None
        if survey.volume:
            n1, n2, n3 = grid.n
            self.vol = torch.empty((6, nf, n3, n2, n1, 2), dtype=torch.float64, device=self.device)


def _check_sigma(grid: Grid, sigma):
    import torch
    if not (isinstance(sigma, torch.Tensor) and sigma.is_cuda and sigma.dtype == torch.float32
            and sigma.is_contiguous()):
        raise TypeError("sigma must be a contiguous CUDA float32 tensor [3][n3][n2][n1]")
    n1, n2, n3 = grid.n
    if tuple(sigma.shape) != (3, n3, n2, n1):
        raise ValueError(f"sigma shape {tuple(sigma.shape)} != (3, {n3}, {n2}, {n1})")


def forward_async(grid: Grid, survey: Survey, sigma, work: Workspace, stream=None) -> None:
    """Enqueue ``emm_forward`` on ``stream`` (default: torch's current stream)
    using the buffers of ``work``; ``sigma`` is a CUDA float32 tensor
    [3][n3][n2][n1]."""
    import torch
    _check_sigma(grid, sigma)
    if stream is None:
        stream = torch.cuda.current_stream(sigma.device)
    s, keep = survey._c()
    code = load_library().emm_forward(
        grid.handle, C.byref(s), C.c_void_p(sigma.data_ptr()), C.c_void_p(work.ptr),
        C.c_size_t(work.bytes), C.c_void_p(work.rec.data_ptr()),
        C.c_void_p(0 if work.vol is None else work.vol.data_ptr()), C.c_void_p(stream.cuda_stream))
    _check(code, "emm_forward")


class WaveWork:
    """Device buffers of ``forward_wave`` for one (grid, survey, depth)."""

    def __init__(self, grid: Grid, survey: Survey, depth: int, device=None):
        import torch
        self.device = torch.device("cuda" if device is None else device)
        s, keep = survey._c()
        n = C.c_size_t(0)
        _check(load_library().emm_wave_workspace_size(grid.handle, C.byref(s), int(depth), C.byref(n)),
               "emm_wave_workspace_size")
        self.depth, self.bytes = int(depth), n.value
        self.ws = torch.empty(self.bytes + 256, dtype=torch.uint8, device=self.device)
        self.ptr = self.ws.data_ptr() + (-self.ws.data_ptr()) % 256
        self.rec = torch.zeros((max(survey.nrec, 1), 6, len(survey.freqs), 2), dtype=torch.float64,
                               device=self.device)


def forward_wave(grid: Grid, survey: Survey, sigma, depth: int = 2, work: Optional[WaveWork] = None,
                 stream=None, check: bool = True):
    """``emm_forward_wave``: the forward solve with ``depth`` time steps in
    flight per sweep of the grid (a persistent launch whose tiles wait on
    per-layer completion counts).  Returns (G complex128 [nrec][6][nfreq],
    work); G equals ``forward``'s bit for bit."""
    import torch
    _check_sigma(grid, sigma)
    if stream is None:
        stream = torch.cuda.current_stream(sigma.device)
    if work is None or work.depth != int(depth):
        work = WaveWork(grid, survey, depth, sigma.device)
    s, keep = survey._c()
    _check(load_library().emm_forward_wave(grid.handle, C.byref(s), C.c_void_p(sigma.data_ptr()), int(depth),
                                           C.c_void_p(work.ptr), C.c_size_t(work.bytes),
                                           C.c_void_p(work.rec.data_ptr()), C.c_void_p(stream.cuda_stream)),
           "emm_forward_wave")
    if check:
        v = C.c_int(0)
        _check(load_library().emm_status(C.c_void_p(work.ptr), C.byref(v), C.c_void_p(stream.cuda_stream)),
               "emm_status")
        if v.value != EMM_OK:
            raise EmmError(v.value, "emm_forward_wave (device status)")
    return torch.view_as_complex(work.rec)[: survey.nrec], work


def forward_converge(grid: Grid, survey: Survey, sigma, work: Workspace, stream=None) -> int:
    """``emm_forward_converge``: ``forward_async`` with the paper's corner
    convergence test every 100 steps (at most ``survey.nt`` steps).
    Synchronous; returns the number of leapfrog steps taken.  ``work.rec``
    (and ``work.vol``) hold the Green's functions of that many steps."""
    import torch
    _check_sigma(grid, sigma)
    if stream is None:
        stream = torch.cuda.current_stream(sigma.device)
    s, keep = survey._c()
    nt_run = C.c_int(0)
    code = load_library().emm_forward_converge(
        grid.handle, C.byref(s), C.c_void_p(sigma.data_ptr()), C.c_void_p(work.ptr),
        C.c_size_t(work.bytes), C.c_void_p(work.rec.data_ptr()),
        C.c_void_p(0 if work.vol is None else work.vol.data_ptr()), C.c_void_p(stream.cuda_stream),
        C.byref(nt_run))
    _check(code, "emm_forward_converge")
    return int(nt_run.value)


def forward_timed(grid: Grid, survey: Survey, sigma, work: Workspace, every: int = 64,
                  stream=None) -> dict:
    """``emm_forward_timed``: like ``forward_async`` but synchronises and
    returns the mean device duration of the E, volume-DTFT and H launches
    (sampled every ``every`` steps), of the time loop and of the whole run,
    in ms."""
    import torch
    _check_sigma(grid, sigma)
    if stream is None:
        stream = torch.cuda.current_stream(sigma.device)
    s, keep = survey._c()
    t = _Timing()
    t.every = int(every)
    code = load_library().emm_forward_timed(
        grid.handle, C.byref(s), C.c_void_p(sigma.data_ptr()), C.c_void_p(work.ptr),
        C.c_size_t(work.bytes), C.c_void_p(work.rec.data_ptr()),
        C.c_void_p(0 if work.vol is None else work.vol.data_ptr()), C.c_void_p(stream.cuda_stream),
        C.byref(t))
    _check(code, "emm_forward_timed")
    return dict(samples=t.samples, e_ms=t.e_ms, h_ms=t.h_ms, v_ms=t.v_ms, total_ms=t.total_ms,
                loop_ms=t.loop_ms)


def forward_static(grid: Grid, survey: Survey, sigma, rec, vol=None, stream=None,
                   wait: bool = True) -> Optional[int]:
    """``emm_forward_static``: the forward run in the library's own static
    device scratch (no device allocation by the call), for callers that may
    not allocate.  ``rec`` (and ``vol`` when ``survey.volume``) are the
    caller's CUDA float64 output tensors, shaped as ``Workspace.rec`` /
    ``Workspace.vol``.  With ``wait`` the call synchronises the stream and
    returns the device status word; otherwise it returns None at once."""
    import torch
    _check_sigma(grid, sigma)
    nf = len(survey.freqs)
    if not (rec.is_cuda and rec.dtype == torch.float64 and rec.is_contiguous()
            and rec.numel() >= max(survey.nrec, 1) * 6 * nf * 2):
        raise TypeError("rec must be a contiguous CUDA float64 tensor [nrec][6][nfreq][2]")
    if survey.volume:
        n1, n2, n3 = grid.n
        if vol is None or not (vol.is_cuda and vol.dtype == torch.float64 and vol.is_contiguous()
                               and vol.numel() == 6 * nf * n1 * n2 * n3 * 2):
            raise TypeError("vol must be a contiguous CUDA float64 tensor [6][nfreq][n3][n2][n1][2]")
    if stream is None:
        stream = torch.cuda.current_stream(sigma.device)
    s, keep = survey._c()
    st = C.c_int(-1)
    code = load_library().emm_forward_static(
        grid.handle, C.byref(s), C.c_void_p(sigma.data_ptr()), C.c_void_p(rec.data_ptr()),
        C.c_void_p(0 if vol is None else vol.data_ptr()), C.c_void_p(stream.cuda_stream),
        C.byref(st) if wait else None)
    _check(code, "emm_forward_static")
    return st.value if wait else None


def batch_workspace_size(grid: Grid, survey: Survey, nsrc: int) -> int:
    """``emm_batch_workspace_size``: device bytes of a batch of nsrc transmitters."""
    s, keep = survey._c()
    n = C.c_size_t(0)
    _check(load_library().emm_batch_workspace_size(grid.handle, C.byref(s), int(nsrc), C.byref(n)),
           "emm_batch_workspace_size")
    return n.value


def forward_batch(grid: Grid, survey: Survey, sigma, src_pos, work=None, stream=None, check: bool = True):
    """``emm_forward_batch``: the receiver Green's functions of several
    transmitters (positions ``src_pos`` [nsrc][3], host) on one conductivity,
    advanced together.  Returns complex128 [nsrc][nrec][6][nfreq] (CUDA) and
    the workspace tensor (pass it back as ``work`` to reuse it)."""
    import torch
    _check_sigma(grid, sigma)
    if stream is None:
        stream = torch.cuda.current_stream(sigma.device)
    pos = _f64(src_pos).reshape(-1, 3)
    nsrc, nf = pos.shape[0], len(survey.freqs)
    s, keep = survey._c()
    nbytes = batch_workspace_size(grid, survey, nsrc)
    if work is None or work.numel() < nbytes + 256:
        work = torch.empty(nbytes + 256, dtype=torch.uint8, device=sigma.device)
    ptr = work.data_ptr() + (-work.data_ptr()) % 256
    rec = torch.zeros((nsrc, max(survey.nrec, 1), 6, nf, 2), dtype=torch.float64, device=sigma.device)
    code = load_library().emm_forward_batch(
        grid.handle, C.byref(s), nsrc, _dp(pos), C.c_void_p(sigma.data_ptr()), C.c_void_p(ptr),
        C.c_size_t(nbytes), C.c_void_p(rec.data_ptr()), C.c_void_p(stream.cuda_stream))
    _check(code, "emm_forward_batch")
    if check:
        v = C.c_int(0)
        _check(load_library().emm_status(C.c_void_p(ptr), C.byref(v), C.c_void_p(stream.cuda_stream)), "emm_status")
        if v.value != EMM_OK:
            raise EmmError(v.value, "emm_forward_batch (device status)")
    return torch.view_as_complex(rec)[:, : survey.nrec], work


def gradient_workspace_size(grid: Grid, survey: Survey, ckpt_every: int, stored_steps: int = 0) -> int:
    s, keep = survey._c()
    n = C.c_size_t(0)
    _check(load_library().emm_gradient_stored_workspace_size(grid.handle, C.byref(s), int(ckpt_every),
                                                             int(stored_steps), C.byref(n)),
           "emm_gradient_stored_workspace_size")
    return n.value


def snapshot_bytes(grid: Grid, survey: Survey, ckpt_every: int) -> int:
    """Device bytes one stored E snapshot adds to the gradient workspace."""
    return (gradient_workspace_size(grid, survey, ckpt_every, 2 * ckpt_every)
            - gradient_workspace_size(grid, survey, ckpt_every, ckpt_every)) // ckpt_every


def vjp(grid: Grid, survey: Survey, sigma, dG, ckpt_every: Optional[int] = None, stream=None, check: bool = True,
        stored_steps: int = 0):
    """``emm_gradient_stored``: the gradient d/dsigma Re(sum conj(dG) G) with
    respect to the interior staggered conductivity (float64 CUDA tensor
    [3][n3][n2][n1]), and G of the forward sweep (complex128
    [nrec][6][nfreq]).  ``dG`` is a complex tensor [nrec][6][nfreq];
    ``ckpt_every`` defaults to about sqrt(nt) steps between checkpoints;
    ``stored_steps`` is the budget of final steps whose E snapshots the
    forward sweep keeps in device memory (whole checkpoint segments), which
    the reverse sweep then does not recompute."""
    import torch
    _check_sigma(grid, sigma)
    if stream is None:
        stream = torch.cuda.current_stream(sigma.device)
    nf = len(survey.freqs)
    if ckpt_every is None:
        ckpt_every = max(1, int(round(max(survey.nt, 1) ** 0.5)))
    nbytes = gradient_workspace_size(grid, survey, ckpt_every, stored_steps)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=sigma.device)
    ptr = ws.data_ptr() + (-ws.data_ptr()) % 256
    dG = torch.as_tensor(dG, dtype=torch.complex128, device=sigma.device).reshape(survey.nrec, 6, nf)
    dG2 = torch.view_as_real(dG.contiguous()).contiguous()
    rec = torch.zeros((max(survey.nrec, 1), 6, nf, 2), dtype=torch.float64, device=sigma.device)
    n1, n2, n3 = grid.n
    grad = torch.empty((3, n3, n2, n1), dtype=torch.float64, device=sigma.device)
    s, keep = survey._c()
    code = load_library().emm_gradient_stored(
        grid.handle, C.byref(s), C.c_void_p(sigma.data_ptr()), C.c_void_p(dG2.data_ptr()), int(ckpt_every),
        int(stored_steps), C.c_void_p(ptr), C.c_size_t(nbytes), C.c_void_p(rec.data_ptr()),
        C.c_void_p(grad.data_ptr()), C.c_void_p(stream.cuda_stream))
    _check(code, "emm_gradient_stored")
    if check:
        v = C.c_int(0)
        _check(load_library().emm_status(C.c_void_p(ptr), C.byref(v), C.c_void_p(stream.cuda_stream)), "emm_status")
        if v.value != EMM_OK:
            raise EmmError(v.value, "emm_gradient (device status)")
    return grad, torch.view_as_complex(rec)[: survey.nrec]


def _emm_function():
    import torch

    class EmmForward(torch.autograd.Function):
        """G = forward(sigma) as a differentiable torch function: the forward
        pass runs ``emm_forward``, the backward pass ``emm_gradient`` with the
        incoming gradient of G as cotangent (torch's convention for a complex
        output of a real input: sigma.grad = Re(sum conj(dG) dG/dsigma))."""

        @staticmethod
        def forward(ctx, sigma, grid, survey, ckpt_every):
            ctx.grid, ctx.survey, ctx.ckpt_every = grid, survey, ckpt_every
            ctx.save_for_backward(sigma)
            G, _ = forward(grid, survey, sigma.detach().to(torch.float32).contiguous())
            return G.clone()

        @staticmethod
        def backward(ctx, dG):
            (sigma,) = ctx.saved_tensors
            grad, _ = vjp(ctx.grid, ctx.survey, sigma.detach().to(torch.float32).contiguous(), dG,
                          ckpt_every=ctx.ckpt_every)
            return grad.to(sigma.dtype), None, None, None

    return EmmForward


def green_functions(sigma, grid: Grid, survey: Survey, ckpt_every: Optional[int] = None):
    """Receiver Green's functions G (complex128 [nrec][6][nfreq]) of the
    conductivity tensor ``sigma`` [3][n3][n2][n1] (CUDA), differentiable with
    respect to ``sigma`` through the exact discrete adjoint."""
    return _emm_function().apply(sigma, grid, survey, ckpt_every)


class Plan:
    """``emm_plan_create`` / ``emm_plan_run``: the time loop of a forward
    solve captured once as a CUDA graph on ``work`` and replayed for each
    conductivity.  ``run(sigma)`` returns (G, vol) like ``forward``."""

    def __init__(self, grid: Grid, survey: Survey, sigma, work: Optional["Workspace"] = None, stream=None):
        import torch
        _check_sigma(grid, sigma)
        self.grid, self.survey = grid, survey
        self.work = work if work is not None else Workspace(grid, survey, sigma.device)
        if stream is None:
            stream = torch.cuda.current_stream(sigma.device)
        s, keep = survey._c()
        h = C.c_void_p()
        vol = self.work.vol.data_ptr() if self.work.vol is not None else None
        _check(load_library().emm_plan_create(grid.handle, C.byref(s), C.c_void_p(sigma.data_ptr()),
                                              C.c_void_p(self.work.ptr), C.c_size_t(self.work.bytes),
                                              C.c_void_p(self.work.rec.data_ptr()), C.c_void_p(vol),
                                              C.c_void_p(stream.cuda_stream), C.byref(h)), "emm_plan_create")
        self._h = h

    def run_async(self, sigma, stream=None):
        import torch
        _check_sigma(self.grid, sigma)
        if stream is None:
            stream = torch.cuda.current_stream(sigma.device)
        _check(load_library().emm_plan_run(self._h, C.c_void_p(sigma.data_ptr()), C.c_void_p(stream.cuda_stream)),
               "emm_plan_run")

    def run(self, sigma, stream=None):
        import torch
        self.run_async(sigma, stream)
        st = status(self.work, stream)
        if st != EMM_OK:
            raise EmmError(st, "emm_plan_run (device status)")
        G = torch.view_as_complex(self.work.rec)[: self.survey.nrec]
        vol = None if self.work.vol is None else torch.view_as_complex(self.work.vol)
        return G, vol

    def close(self):
        """``emm_plan_destroy`` now (otherwise when the object is collected)."""
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.emm_plan_destroy(h)
        self._h = None

    def __del__(self):
        self.close()


class JobsWork:
    """Workspace of ``forward_jobs`` for a fixed list of (grid, survey)
    problems: the device buffer, each problem's offset in it and its
    receiver output."""

    def __init__(self, problems, device="cuda"):
        import torch
        self.problems = list(problems)
        jobs, self._keep = _jobs_c(self.problems, [None] * len(self.problems), [None] * len(self.problems))
        n = C.c_size_t(0)
        offs = (C.c_size_t * len(jobs))()
        _check(load_library().emm_jobs_workspace_size(len(jobs), jobs, C.byref(n), offs), "emm_jobs_workspace_size")
        self.nbytes = n.value
        self.buf = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=device)
        self.ptr = self.buf.data_ptr() + (-self.buf.data_ptr()) % 256
        self.offsets = [int(o) for o in offs]
        self.strategy, self.tune_ms = None, None
        self.rec = [torch.zeros((max(s.nrec, 1), 6, len(s.freqs), 2), dtype=torch.float64, device=device)
                    for _, s in self.problems]

    def status(self, stream=None):
        """Device status word of each problem of the last run (synchronises)."""
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(self.buf.device)
        out = []
        for off in self.offsets:
            v = C.c_int(0)
            _check(load_library().emm_status(C.c_void_p(self.ptr + off), C.byref(v), C.c_void_p(stream.cuda_stream)),
                   "emm_status")
            out.append(int(v.value))
        return out


def _jobs_c(problems, sigmas, recs):
    jobs = (_Job * len(problems))()
    keep = []
    for j, (grid, survey) in enumerate(problems):
        sc, k = survey._c()
        keep += [sc, k]
        jobs[j].grid = grid.handle
        jobs[j].survey = C.pointer(sc)
        jobs[j].sigma = sigmas[j].data_ptr() if sigmas[j] is not None else None
        jobs[j].rec_out = recs[j].data_ptr() if recs[j] is not None else None
    return jobs, keep


def jobs_tune(problems, sigmas, work: "JobsWork", steps: int = 40, stream=None):
    """``emm_jobs_tune``: times ``steps`` leapfrog steps of ``problems`` by
    each strategy and returns (best strategy, {name: ms})."""
    import torch
    dev = sigmas[0].device
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    jobs, keep = _jobs_c(list(problems), list(sigmas), work.rec)
    ms = np.zeros(3)
    best = C.c_int(0)
    _check(load_library().emm_jobs_tune(len(jobs), jobs, C.c_void_p(work.ptr), C.c_size_t(work.nbytes), int(steps),
                                        C.c_void_p(stream.cuda_stream), _dp(ms), C.byref(best)), "emm_jobs_tune")
    return int(best.value), dict(zip(JOBS_STRATEGIES, ms.tolist()))


def forward_jobs(problems, sigmas, work: Optional[JobsWork] = None, stream=None, check: bool = True,
                 strategy: Optional[int] = None):
    """``emm_forward_jobs``: the forward solves of ``problems`` (a list of
    (Grid, Survey), up to 16, one FD order) advanced together by
    ``strategy`` (JOBS_LIST, JOBS_SEQUENTIAL or JOBS_STREAMS; None: the one
    ``jobs_tune`` finds fastest, tuned once per ``work``).  ``sigmas`` are
    float32 CUDA tensors [3][n3][n2][n1].  Returns ([G complex128
    [nrec][6][nfreq] per problem], work)."""
    import torch
    problems = list(problems)
    for (grid, _), sg in zip(problems, sigmas):
        _check_sigma(grid, sg)
    dev = sigmas[0].device
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    if work is None:
        work = JobsWork(problems, dev)
    if strategy is None:
        if work.strategy is None:
            work.strategy, work.tune_ms = jobs_tune(problems, sigmas, work, stream=stream)
        strategy = work.strategy
    jobs, keep = _jobs_c(problems, list(sigmas), work.rec)
    _check(load_library().emm_forward_jobs(len(jobs), jobs, int(strategy), C.c_void_p(work.ptr),
                                           C.c_size_t(work.nbytes), C.c_void_p(stream.cuda_stream)),
           "emm_forward_jobs")
    if check:
        for j, v in enumerate(work.status(stream)):
            if v != EMM_OK:
                raise EmmError(v, f"emm_forward_jobs (device status of problem {j})")
    return [torch.view_as_complex(r)[: s.nrec] for r, (_, s) in zip(work.rec, problems)], work


class PersistWork:
    """Workspace and outputs of the persistent work list for fixed tasks.
    A task is (Grid, Survey, src_pos): ``src_pos`` None (the survey's
    transmitter) or [nsrc][3] transmitters sharing grid and conductivity.
    ``rec[j]`` is task j's float64 output [nsrc][nrec][6][nfreq][2]."""

    def __init__(self, tasks, device="cuda"):
        import torch
        self.tasks = [(g, s, None if p is None else np.ascontiguousarray(p, dtype=np.float64).reshape(-1, 3))
                      for g, s, p in tasks]
        self.rec = [torch.zeros((1 if p is None else len(p), max(s.nrec, 1), 6, len(s.freqs), 2),
                                dtype=torch.float64, device=device) for _, s, p in self.tasks]
        arr, self._keep = self._c([None] * len(self.tasks))
        n = C.c_size_t(0)
        offs = (C.c_size_t * len(self.tasks))()
        _check(load_library().emm_persist_workspace_size(len(self.tasks), arr, C.byref(n), offs),
               "emm_persist_workspace_size")
        self.nbytes = n.value
        self.buf = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=device)
        self.ptr = self.buf.data_ptr() + (-self.buf.data_ptr()) % 256
        self.offsets = [int(o) for o in offs]
        self.best, self.tune_ms = None, None

    def _c(self, sigmas):
        arr = (_Task * len(self.tasks))()
        keep = []
        for j, (grid, survey, pos) in enumerate(self.tasks):
            sc, k = survey._c()
            keep += [sc, k]
            arr[j].grid = grid.handle
            arr[j].survey = C.pointer(sc)
            arr[j].sigma = sigmas[j].data_ptr() if sigmas[j] is not None else None
            arr[j].nsrc = 1 if pos is None else len(pos)
            arr[j].src_pos = _dp(pos) if pos is not None else None
            arr[j].rec_out = self.rec[j].data_ptr()
        return arr, keep

    def _status_at(self, off, stream):
        v = C.c_int(0)
        _check(load_library().emm_status(C.c_void_p(self.ptr + off), C.byref(v), C.c_void_p(stream.cuda_stream)),
               "emm_status")
        return int(v.value)

    def status(self, stream=None):
        """(work-list status, [each task's status]) of the last run
        (synchronises)."""
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(self.buf.device)
        return self._status_at(0, stream), [self._status_at(o, stream) for o in self.offsets]

    def G(self):
        """Each task's Green's functions, complex128 [nsrc][nrec][6][nfreq]."""
        import torch
        return [torch.view_as_complex(r)[:, : s.nrec] for r, (_, s, _) in zip(self.rec, self.tasks)]


def _persist_check(work: PersistWork, sigmas):
    sigmas = list(sigmas)
    if len(sigmas) != len(work.tasks):
        raise ValueError("one sigma per task")
    for (grid, _, _), sg in zip(work.tasks, sigmas):
        _check_sigma(grid, sg)
    return sigmas


def persist_tune(work: PersistWork, sigmas, steps: int = 40, candidates: int = 16, stream=None):
    """``emm_persist_tune``: times ``steps`` leapfrog steps of each tile
    shape with 1, 2, ... resident CTAs per SM and returns (best PersistOpts,
    {(tile_shape, ctas_per_sm): ms})."""
    import torch
    sigmas = _persist_check(work, sigmas)
    if stream is None:
        stream = torch.cuda.current_stream(sigmas[0].device)
    arr, keep = work._c(sigmas)
    ms = np.zeros(int(candidates))
    cands = (PersistOpts * int(candidates))()
    nc = C.c_int(int(candidates))
    best = PersistOpts()
    _check(load_library().emm_persist_tune(len(work.tasks), arr, C.c_void_p(work.ptr), C.c_size_t(work.nbytes),
                                           int(steps), C.c_void_p(stream.cuda_stream), C.byref(nc), cands, _dp(ms),
                                           C.byref(best)), "emm_persist_tune")
    return best, {cands[k].key(): float(ms[k]) for k in range(nc.value)}


def forward_persistent(work: PersistWork, sigmas, opts: Optional[PersistOpts] = None, stream=None,
                       check: bool = True):
    """``emm_forward_persistent``: every task's forward solve in one
    persistent cooperative launch.  ``opts`` None: the options
    ``persist_tune`` finds fastest (tuned once per ``work``).  Returns each
    task's G (complex128 [nsrc][nrec][6][nfreq]); with ``check`` the status
    words are read (synchronises) and a failure raises."""
    import torch
    sigmas = _persist_check(work, sigmas)
    if stream is None:
        stream = torch.cuda.current_stream(sigmas[0].device)
    if opts is None:
        if work.best is None:
            work.best, work.tune_ms = persist_tune(work, sigmas, stream=stream)
        opts = work.best
    arr, keep = work._c(sigmas)
    _check(load_library().emm_forward_persistent(len(work.tasks), arr, C.byref(opts), C.c_void_p(work.ptr),
                                                 C.c_size_t(work.nbytes), C.c_void_p(stream.cuda_stream)),
           "emm_forward_persistent")
    if check:
        top, each = work.status(stream)
        if top != EMM_OK:
            raise EmmError(top, "emm_forward_persistent (work-list status)")
        for j, v in enumerate(each):
            if v != EMM_OK:
                raise EmmError(v, f"emm_forward_persistent (device status of task {j})")
    return work.G()


class PersistPlan:
    """``emm_persist_plan_create`` / ``_run``: the persistent solve of
    ``work``'s tasks on the buffers ``sigmas`` captured once as a CUDA graph;
    ``run()`` replays it for their current contents."""

    def __init__(self, work: PersistWork, sigmas, opts: Optional[PersistOpts] = None, stream=None):
        import torch
        self.work = work
        self.sigmas = _persist_check(work, sigmas)
        if stream is None:
            stream = torch.cuda.current_stream(self.sigmas[0].device)
        arr, keep = work._c(self.sigmas)
        h = C.c_void_p()
        _check(load_library().emm_persist_plan_create(len(work.tasks), arr,
                                                      C.byref(opts) if opts is not None else None,
                                                      C.c_void_p(work.ptr), C.c_size_t(work.nbytes),
                                                      C.c_void_p(stream.cuda_stream), C.byref(h)),
               "emm_persist_plan_create")
        self._h = h

    def run_async(self, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(self.sigmas[0].device)
        _check(load_library().emm_persist_plan_run(self._h, C.c_void_p(stream.cuda_stream)), "emm_persist_plan_run")

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.emm_persist_plan_destroy(h)
        self._h = None

    def __del__(self):
        self.close()


def _stagger_ws(grid: Grid, device):
    import torch
    n = C.c_size_t(0)
    _check(load_library().emm_stagger_workspace_size(grid.handle, C.byref(n)), "emm_stagger_workspace_size")
    return torch.empty(max(1, (n.value + 7) // 8), dtype=torch.float64, device=device)


def _cells_shape(grid: Grid):
    n1, n2, n3 = grid.n
    return (n3 - 1, n2 - 1, n1 - 1)


def stagger_sigma(grid: Grid, sigma_h, sigma_v, stream=None):
    """``emm_stagger_sigma``: the staggered conductivity (float32 CUDA tensor
    [3][n3][n2][n1], what ``forward`` takes) from cell-centred sigma_h and
    sigma_v (float64 CUDA tensors [n3-1][n2-1][n1-1]): face-area weighted
    means over the cells around each edge (Sec. 3.6)."""
    import torch
    sh = torch.as_tensor(sigma_h, dtype=torch.float64, device="cuda").contiguous()
    sv = torch.as_tensor(sigma_v, dtype=torch.float64, device=sh.device).contiguous()
    if tuple(sh.shape) != _cells_shape(grid) or tuple(sv.shape) != _cells_shape(grid):
        raise ValueError(f"cell arrays must have shape {_cells_shape(grid)}")
    if stream is None:
        stream = torch.cuda.current_stream(sh.device)
    n1, n2, n3 = grid.n
    out = torch.empty((3, n3, n2, n1), dtype=torch.float32, device=sh.device)
    ws = _stagger_ws(grid, sh.device)
    _check(load_library().emm_stagger_sigma(grid.handle, C.c_void_p(sh.data_ptr()), C.c_void_p(sv.data_ptr()),
                                            C.c_void_p(ws.data_ptr()), C.c_size_t(ws.numel() * 8),
                                            C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream)),
           "emm_stagger_sigma")
    return out


def stagger_sigma_adjoint(grid: Grid, grad, grad_h=None, grad_v=None, stream=None):
    """``emm_stagger_sigma_adjoint``: adds the transpose of ``stagger_sigma``
    applied to ``grad`` (float64 CUDA [3][n3][n2][n1]) to ``grad_h`` and
    ``grad_v`` (float64 CUDA [n3-1][n2-1][n1-1]; zeros if not given) and
    returns them."""
    import torch
    grad = grad.contiguous()
    if stream is None:
        stream = torch.cuda.current_stream(grad.device)
    if grad_h is None:
        grad_h = torch.zeros(_cells_shape(grid), dtype=torch.float64, device=grad.device)
    if grad_v is None:
        grad_v = torch.zeros(_cells_shape(grid), dtype=torch.float64, device=grad.device)
    ws = _stagger_ws(grid, grad.device)
    _check(load_library().emm_stagger_sigma_adjoint(grid.handle, C.c_void_p(grad.data_ptr()),
                                                    C.c_void_p(ws.data_ptr()), C.c_size_t(ws.numel() * 8),
                                                    C.c_void_p(grad_h.data_ptr()), C.c_void_p(grad_v.data_ptr()),
                                                    C.c_void_p(stream.cuda_stream)),
           "emm_stagger_sigma_adjoint")
    return grad_h, grad_v


class GradientWork:
    """Device buffers of ``misfit_gradient`` (workspace, G and the gradient),
    kept between the transmitters of a survey."""

    def __init__(self, grid: Grid, survey: Survey, ckpt_every: int, stored_steps: int = 0, device="cuda"):
        import torch
        self.ckpt_every, self.stored_steps = int(ckpt_every), int(stored_steps)
        self.nbytes = gradient_workspace_size(grid, survey, self.ckpt_every, self.stored_steps)
        self.buf = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=device)
        self.ptr = self.buf.data_ptr() + (-self.buf.data_ptr()) % 256
        n1, n2, n3 = grid.n
        self.rec = torch.zeros((max(survey.nrec, 1), 6, len(survey.freqs), 2), dtype=torch.float64, device=device)
        self.grad = torch.empty((3, n3, n2, n1), dtype=torch.float64, device=device)


def misfit_gradient(grid: Grid, survey: Survey, sigma, d_obs, weight=None, ckpt_every: Optional[int] = None,
                    stored_steps: int = 0, misfit=None, work: Optional[GradientWork] = None, stream=None,
                    check: bool = True):
    """``emm_misfit_gradient`` for one transmitter: adds 1/2 sum w |G - d_obs|^2
    to ``misfit`` (float64 CUDA tensor [1], zeros if not given) and returns
    (misfit, grad, G), grad the float64 [3][n3][n2][n1] gradient with respect
    to the staggered conductivity, G complex128 [nrec][6][nfreq].  ``d_obs``
    is complex [nrec][6][nfreq], ``weight`` real [nrec][6][nfreq] or None."""
    import torch
    _check_sigma(grid, sigma)
    dev = sigma.device
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    nf = len(survey.freqs)
    if ckpt_every is None:
        ckpt_every = max(1, int(round(max(survey.nt, 1) ** 0.5)))
    if work is None or work.ckpt_every != ckpt_every or work.stored_steps != stored_steps:
        work = GradientWork(grid, survey, ckpt_every, stored_steps, dev)
    d = torch.as_tensor(d_obs, dtype=torch.complex128, device=dev).reshape(survey.nrec, 6, nf)
    d2 = torch.view_as_real(d.contiguous()).contiguous()
    w = None
    if weight is not None:
        w = torch.as_tensor(weight, dtype=torch.float64, device=dev).reshape(survey.nrec, 6, nf).contiguous()
    if misfit is None:
        misfit = torch.zeros(1, dtype=torch.float64, device=dev)
    s, keep = survey._c()
    code = load_library().emm_misfit_gradient(
        grid.handle, C.byref(s), C.c_void_p(sigma.data_ptr()), C.c_void_p(d2.data_ptr()),
        C.c_void_p(w.data_ptr() if w is not None else None), int(ckpt_every), int(stored_steps),
        C.c_void_p(work.ptr), C.c_size_t(work.nbytes), C.c_void_p(work.rec.data_ptr()), C.c_void_p(misfit.data_ptr()),
        C.c_void_p(work.grad.data_ptr()), C.c_void_p(stream.cuda_stream))
    _check(code, "emm_misfit_gradient")
    if check:
        v = C.c_int(0)
        _check(load_library().emm_status(C.c_void_p(work.ptr), C.byref(v), C.c_void_p(stream.cuda_stream)),
               "emm_status")
        if v.value != EMM_OK:
            raise EmmError(v.value, "emm_misfit_gradient (device status)")
    return misfit, work.grad, torch.view_as_complex(work.rec)[: survey.nrec]


def survey_misfit_gradient(grid: Grid, survey: Survey, sigma_h, sigma_v, src_pos, d_obs, weight=None,
                           ckpt_every: Optional[int] = None, stored_steps: int = 0, stream=None,
                           check: bool = True):
    """Least-squares misfit of a survey and its gradient with respect to the
    cell conductivities: for every transmitter position in ``src_pos``
    ([nsrc][3], the rest of ``survey`` shared) one ``emm_misfit_gradient``,
    whose gradient ``emm_stagger_sigma_adjoint`` adds to the cells.  Returns
    (misfit float64 CUDA [1], grad_h, grad_v float64 CUDA [n3-1][n2-1][n1-1],
    G complex128 [nsrc][nrec][6][nfreq]).  ``d_obs`` is [nsrc][nrec][6][nfreq],
    ``weight`` None, [nrec][6][nfreq] (shared) or [nsrc][nrec][6][nfreq]."""
    import torch
    sigma = stagger_sigma(grid, sigma_h, sigma_v, stream)
    dev = sigma.device
    pos = np.asarray(src_pos, dtype=np.float64).reshape(-1, 3)
    if ckpt_every is None:
        ckpt_every = max(1, int(round(max(survey.nt, 1) ** 0.5)))
    work = GradientWork(grid, survey, ckpt_every, stored_steps, dev)
    misfit = torch.zeros(1, dtype=torch.float64, device=dev)
    grad_h = torch.zeros(_cells_shape(grid), dtype=torch.float64, device=dev)
    grad_v = torch.zeros(_cells_shape(grid), dtype=torch.float64, device=dev)
    Gs = []
    w_all = None if weight is None else torch.as_tensor(weight, dtype=torch.float64)
    for k, p in enumerate(pos):
        sk = dataclasses.replace(survey, src=tuple(float(v) for v in p))
        wk = None if w_all is None else (w_all[k] if w_all.dim() == 4 else w_all)
        _, grad, G = misfit_gradient(grid, sk, sigma, d_obs[k], wk, ckpt_every, stored_steps, misfit, work,
                                     stream, check)
        stagger_sigma_adjoint(grid, grad, grad_h, grad_v, stream)
        Gs.append(G.clone())
    return misfit, grad_h, grad_v, torch.stack(Gs)


def _cell_misfit_function():
    import torch

    class CellMisfit(torch.autograd.Function):
        """The survey misfit as a differentiable function of the cell
        conductivities sigma_h, sigma_v: the forward pass runs
        ``survey_misfit_gradient`` (forward sweeps, residuals, adjoint sweeps)
        and keeps the gradient, which the backward pass scales by the
        incoming gradient of the scalar misfit."""

        @staticmethod
        def forward(ctx, sigma_h, sigma_v, grid, survey, src_pos, d_obs, weight, ckpt_every, stored_steps):
            misfit, gh, gv, _ = survey_misfit_gradient(grid, survey, sigma_h.detach(), sigma_v.detach(), src_pos,
                                                       d_obs, weight, ckpt_every, stored_steps)
            ctx.save_for_backward(gh, gv)
            return misfit[0].clone()

        @staticmethod
        def backward(ctx, g):
            gh, gv = ctx.saved_tensors
            return (g * gh).to(gh.dtype), (g * gv).to(gv.dtype), None, None, None, None, None, None, None

    return CellMisfit


def cell_misfit(sigma_h, sigma_v, grid: Grid, survey: Survey, src_pos, d_obs, weight=None,
                ckpt_every: Optional[int] = None, stored_steps: int = 0):
    """Survey misfit 1/2 sum w |G - d_obs|^2 (float64 CUDA scalar) of the cell
    conductivities, differentiable with respect to ``sigma_h`` and
    ``sigma_v`` (float64 CUDA [n3-1][n2-1][n1-1])."""
    return _cell_misfit_function().apply(sigma_h, sigma_v, grid, survey, src_pos, d_obs, weight, ckpt_every,
                                         stored_steps)


def status(work: Workspace, stream=None) -> int:
    """Device status word of the last forward run on ``work`` (synchronises)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(work.device)
    st = C.c_int()
    _check(load_library().emm_status(C.c_void_p(work.ptr), C.byref(st), C.c_void_p(stream.cuda_stream)),
           "emm_status")
    return int(st.value)


def forward(grid: Grid, survey: Survey, sigma, work: Optional[Workspace] = None, check: bool = True):
    """Run one forward solve and return (G, vol) as complex128 torch tensors on
    the GPU (``vol`` is None unless ``survey.volume``).  ``sigma`` may be a
    numpy array or a CPU tensor; it is copied to the GPU first."""
    import torch
    if not isinstance(sigma, torch.Tensor):
        sigma = torch.from_numpy(np.ascontiguousarray(sigma, dtype=np.float32))
    if not sigma.is_cuda:
        sigma = sigma.to(device="cuda", dtype=torch.float32, non_blocking=True)
    sigma = sigma.contiguous()
    if work is None:
        work = Workspace(grid, survey, sigma.device)
    forward_async(grid, survey, sigma, work)
    if check:
        st = status(work)
        if st != EMM_OK:
            raise EmmError(st, "emm_forward (device status)")
    G = torch.view_as_complex(work.rec)[: survey.nrec]
    vol = None if work.vol is None else torch.view_as_complex(work.vol)
    return G, vol


def survey_for(workload, nt: Optional[int] = None, dt: float = 0.0, **kw) -> Survey:
    """Survey of a :class:`workloads.Workload` (sigma_min from its model)."""
    nt = workload.nt if nt is None else nt
    if nt is None:
        raise ValueError("nt required (the workload fixes only t_max)")
    args = dict(omega0=workload.omega0, fmax=workload.fmax,
                sigma_min=float(np.min(workload.sigma)), nt=int(nt), src=tuple(workload.src),
                rec=workload.rec, freqs=tuple(workload.freqs), dt=dt, src_az=workload.src_az,
                src_dip=workload.src_dip, moment=workload.moment, volume=workload.volume)
    args.update(kw)
    return Survey(**args)


def grid_for(workload) -> Grid:
    return Grid(workload.x, workload.y, workload.z, workload.rd, workload.nb, workload.ne)


def steps_for(workload, grid: Optional[Grid] = None) -> int:
    """ceil(t_max / dt) with dt = 0.99/eta of the workload's grid and model."""
    if workload.nt is not None:
        return int(workload.nt)
    grid = grid_for(workload) if grid is None else grid
    dt, _, _ = grid.time_step(float(np.min(workload.sigma)), workload.omega0)
    return int(math.ceil(workload.t_max / dt))
