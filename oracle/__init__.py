"""FP64 CPU oracle of the fictitious-wave FDTD method (test infrastructure).

The oracle is the slow, plain reference every CUDA result is checked against.
Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA library: the C
source ``emm_oracle.c`` is written independently from the paper (Yang, libEMM,
arXiv 2304.00233) and this module only marshals arrays through ctypes.

Entry points:
  * ``build()``       compile ``emm_oracle.c`` with gcc (FP64, OpenMP, no FMA
                      contraction) into ``oracle/_build/liboracle.so``.
  * ``row_weights``   row 0 / row 1 of [V^T]^{-1}  (Sec. 3.1, Eq. 9-12).
  * ``vander_inverse``full [V^T]^{-1} by unit vectors (Eq. 12).
  * ``vjp``           exact discrete adjoint of ``forward`` (gradient of
                      Re(sum conj(v) G) with respect to the conductivity).
  * ``axis_tables``   padded nodes, half nodes, D+/D- rows, CPML slabs and
                      coefficients, D_max  (Sec. 3.1-3.4).
  * ``locate``        source/receiver stencil start and 1-D weights.
  * ``forward``       the whole time loop of Algorithm 1 (no airwave) and the
                      Green's functions of Eq. 7.
  * ``stagger`` / ``stagger_T``  staggered conductivity from cell sigma_h,
                      sigma_v (Sec. 3.6) and its transpose.
  * ``misfit_gradient`` least-squares misfit of receiver data and its
                      gradient with respect to the cell conductivities
                      (``forward``, the residual, ``vjp``, ``stagger_T``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Dict, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "emm_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

ERRORS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "outside interior"}


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, OpenMP, -ffp-contract=off)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
           "-std=gnu11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        D = C.POINTER(C.c_double)
        I = C.POINTER(C.c_int)
        _lib.orc_vander_inverse.argtypes = [C.c_int, D, D]
        _lib.orc_row_weights.argtypes = [C.c_int, D, C.c_double, C.c_int, D]
        _lib.orc_axis_tables.argtypes = [C.c_int, D, C.c_int, C.c_int, C.c_int,
                                         C.c_double, C.c_double, C.c_double,
                                         D, D, D, D, I, I, D, D, I]
        _lib.orc_axis_tables.restype = C.c_int
        _lib.orc_locate.argtypes = [C.c_int, D, C.c_int, D, C.c_int, D, C.c_int,
                                    C.c_int, C.c_int, C.c_int, D, I, D]
        _lib.orc_locate.restype = C.c_int
        _lib.orc_forward.argtypes = [C.POINTER(_Problem)]
        _lib.orc_forward.restype = C.c_int
        _lib.orc_vjp.argtypes = [C.POINTER(_Problem), D, D, C.c_int]
        _lib.orc_vjp.restype = C.c_int
        _lib.orc_threads.restype = C.c_int
        _lib.orc_stagger.argtypes = [I, C.POINTER(D), D, D, D]
        _lib.orc_stagger.restype = C.c_int
        _lib.orc_stagger_T.argtypes = [I, C.POINTER(D), D, D, D]
        _lib.orc_stagger_T.restype = C.c_int
    return _lib


def threads() -> int:
    """OpenMP threads the oracle's loops use."""
    return int(_load().orc_threads())


def _dp(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleError(RuntimeError):
    pass


def _check(code: int, what: str):
    if code != 0:
        raise OracleError(f"{what}: {ERRORS.get(code, code)}")


def vander_inverse(t) -> np.ndarray:
    t = _f64(t)
    m = len(t)
    W = np.zeros((m, m))
    _load().orc_vander_inverse(m, _dp(t), _dp(W))
    return W


def row_weights(knots, x: float, row: int) -> np.ndarray:
    knots = _f64(knots)
    w = np.zeros(len(knots))
    _load().orc_row_weights(len(knots), _dp(knots), float(x), int(row), _dp(w))
    return w


def axis_tables(x, rd: int, nb: int, ne: int, vmax: float = 1.0,
                fmax: float = 1.0, dt: float = 1.0) -> Dict[str, np.ndarray]:
    x = _f64(x)
    n = len(x)
    npad = n + 2 * (nb + ne)
    m = 2 * rd
    out = dict(X=np.zeros(npad + 1), Xh=np.zeros(npad), cp=np.zeros((npad, m)),
               cm=np.zeros((npad, m)), slab=np.zeros(npad, np.int32),
               slabh=np.zeros(npad, np.int32),
               pml=np.zeros((4, 2 * nb)), dmax=np.zeros(1), ranges=np.zeros(4, np.int32))
    code = _load().orc_axis_tables(n, _dp(x), rd, nb, ne, vmax, fmax, dt,
                                   _dp(out["X"]), _dp(out["Xh"]), _dp(out["cp"]),
                                   _dp(out["cm"]), _ip(out["slab"]), _ip(out["slabh"]),
                                   _dp(out["pml"]),
                                   _dp(out["dmax"]), _ip(out["ranges"]))
    _check(code, "axis_tables")
    out["dmax"] = float(out["dmax"][0])
    return out


def locate(x, y, z, rd: int, nb: int, ne: int, comp: int, pos):
    """Stencil start (i,j,k of the first knot) and 1-D weights [3][2rd] of
    component ``comp`` (0..5 = Ex Ey Ez Hx Hy Hz) at ``pos``."""
    x, y, z, pos = _f64(x), _f64(y), _f64(z), _f64(pos)
    start = np.zeros(3, np.int32)
    w = np.zeros((3, 2 * rd))
    code = _load().orc_locate(len(x), _dp(x), len(y), _dp(y), len(z), _dp(z),
                              rd, nb, ne, comp, _dp(pos), _ip(start), _dp(w))
    _check(code, "locate")
    return start, w


class _Problem(C.Structure):
    _fields_ = [
        ("n", C.c_int * 3),
        ("x", C.POINTER(C.c_double) * 3),
        ("rd", C.c_int), ("nb", C.c_int), ("ne", C.c_int),
        ("sigma", C.POINTER(C.c_double)),
        ("omega0", C.c_double), ("sigma_min", C.c_double), ("dt", C.c_double),
        ("nt", C.c_int), ("fmax", C.c_double),
        ("src", C.c_double * 3),
        ("az", C.c_double), ("dip", C.c_double), ("moment", C.c_double),
        ("nrec", C.c_int), ("rec", C.POINTER(C.c_double)),
        ("nfreq", C.c_int), ("freqs", C.POINTER(C.c_double)),
        ("want_volume", C.c_int), ("convergence", C.c_int),
        ("inject", C.c_int), ("pml", C.c_int),
        ("init_fields", C.POINTER(C.c_double)),
        ("final_fields", C.POINTER(C.c_double)),
        ("rec_G", C.POINTER(C.c_double)), ("rec_acc", C.POINTER(C.c_double)),
        ("jhat", C.POINTER(C.c_double)), ("vol_G", C.POINTER(C.c_double)),
        ("info", C.POINTER(C.c_double)),
        ("nvs", C.c_int), ("vs_idx", C.POINTER(C.c_longlong)),
        ("vs_G", C.POINTER(C.c_double)),
        ("magnetic", C.c_int),
        ("src_length", C.c_double), ("src_points", C.c_int),
        ("airwave", C.c_int),
    ]


def forward(x, y, z, sigma, *, rd: int, nb: int, ne: int, omega0: float,
            nt: int, fmax: float, src=(0.0, 0.0, 0.0), az: float = 0.0,
            dip: float = 0.0, moment: float = 1.0, rec=None, freqs=(),
            sigma_min: float = 0.0, dt: float = 0.0, volume: bool = False,
            convergence: bool = False, inject: bool = True, pml: bool = True,
            init_fields: Optional[np.ndarray] = None,
            want_fields: bool = False,
            vol_samples: Optional[np.ndarray] = None,
            magnetic: bool = False, src_length: float = 0.0,
            src_points: int = 1, airwave: bool = False) -> Dict[str, object]:
    """Run the FP64 oracle.  ``sigma`` is [3][n3][n2][n1] (staggered sigma_xx,
    sigma_yy, sigma_zz).  Returns a dict with ``G`` [nrec][6][nfreq] complex,
    ``acc`` (raw DTFT), ``jhat`` [nfreq], optional ``vol`` [6][nfreq][n3][n2][n1]
    and ``fields`` [6][n3p][n2p][n1p], plus ``dt``, ``vmax``, ``nt``, ``eta``.
    ``vol_samples`` (flat indices into [6][n3][n2][n1]) gives ``vol_samples_G``
    [nvs][nfreq]: the volume Green's functions at those samples only.
    ``magnetic``: the dipole is a magnetic source M (G^EH, G^HH) instead of an
    electric current J (G^EE, G^HE).  ``src_length`` > 0: an antenna of that
    length along the dipole direction, centred at ``src``, as ``src_points``
    equal sub-dipoles at the midpoints of equal segments.  ``airwave``: air
    above the top interior node (needs uniform x and y)."""
    lib = _load()
    xs = [_f64(x), _f64(y), _f64(z)]
    n = [len(a) for a in xs]
    npad = [k + 2 * (nb + ne) for k in n]
    sigma = _f64(sigma)
    assert sigma.shape == (3, n[2], n[1], n[0]), sigma.shape
    rec = _f64(np.zeros((0, 3)) if rec is None else rec).reshape(-1, 3)
    freqs = _f64(freqs)
    nrec, nf = rec.shape[0], len(freqs)
    P = _Problem()
    P.n = (C.c_int * 3)(*n)
    P.x = (C.POINTER(C.c_double) * 3)(*[_dp(a) for a in xs])
    P.rd, P.nb, P.ne = rd, nb, ne
    P.sigma = _dp(sigma)
    P.omega0, P.sigma_min, P.dt = omega0, sigma_min, dt
    P.nt, P.fmax = int(nt), fmax
    P.src = (C.c_double * 3)(*[float(v) for v in src])
    P.az, P.dip, P.moment = az, dip, moment
    P.nrec = nrec
    P.rec = _dp(rec) if nrec else None
    P.nfreq = nf
    P.freqs = _dp(freqs) if nf else None
    P.want_volume = int(volume)
    P.convergence = int(convergence)
    P.inject, P.pml = int(inject), int(pml)
    P.magnetic = int(magnetic)
    P.src_length, P.src_points = float(src_length), int(src_points)
    P.airwave = int(airwave)
    ncell = npad[0] * npad[1] * npad[2]
    if init_fields is not None:
        init_fields = _f64(init_fields)
        assert init_fields.size == 6 * ncell
        P.init_fields = _dp(init_fields)
    fields = np.zeros((6, npad[2], npad[1], npad[0])) if want_fields else None
    P.final_fields = _dp(fields)
    G = np.zeros((max(nrec, 1), 6, max(nf, 1), 2))
    acc = np.zeros_like(G)
    jh = np.zeros((max(nf, 1), 2))
    vol = np.zeros((6, nf, n[2], n[1], n[0], 2)) if volume else None
    info = np.zeros(4)
    P.rec_G, P.rec_acc, P.jhat, P.vol_G, P.info = _dp(G), _dp(acc), _dp(jh), _dp(vol), _dp(info)
    vsG = None
    if vol_samples is not None:
        vs = np.ascontiguousarray(vol_samples, dtype=np.int64)
        P.nvs = len(vs)
        P.vs_idx = vs.ctypes.data_as(C.POINTER(C.c_longlong))
        vsG = np.zeros((len(vs), max(nf, 1), 2))
        P.vs_G = _dp(vsG)
    code = lib.orc_forward(C.byref(P))
    _check(code, "forward")
    cplx = lambda a: a[..., 0] + 1j * a[..., 1]
    out = dict(G=cplx(G)[:nrec, :, :nf], acc=cplx(acc)[:nrec, :, :nf], jhat=cplx(jh)[:nf],
               dt=float(info[0]), vmax=float(info[1]), nt=int(info[2]), eta=float(info[3]))
    if volume:
        out["vol"] = cplx(vol)
    if want_fields:
        out["fields"] = fields
    if vsG is not None:
        out["vol_samples_G"] = cplx(vsG)[:, :nf]
    return out


def vjp(x, y, z, sigma, v, *, rd: int, nb: int, ne: int, omega0: float, nt: int,
        fmax: float, sigma_min: float, src=(0.0, 0.0, 0.0), az: float = 0.0,
        dip: float = 0.0, moment: float = 1.0, rec=None, freqs=(), dt: float = 0.0,
        inject: bool = True, pml: bool = True, ckpt_every: int = 50) -> np.ndarray:
    """Exact discrete adjoint of ``forward``: the gradient with respect to the
    interior staggered conductivity [3][n3][n2][n1] of Re(sum conj(v) G),
    ``v`` a complex cotangent [nrec][6][nfreq] of the receiver Green's
    functions.  ``sigma_min`` (> 0) and ``dt`` fix the time step and the CPML
    as ``forward`` would with the same arguments."""
    lib = _load()
    xs = [_f64(x), _f64(y), _f64(z)]
    n = [len(a) for a in xs]
    sigma = _f64(sigma)
    assert sigma.shape == (3, n[2], n[1], n[0]), sigma.shape
    rec = _f64(np.zeros((0, 3)) if rec is None else rec).reshape(-1, 3)
    freqs = _f64(freqs)
    nrec, nf = rec.shape[0], len(freqs)
    v = np.asarray(v, dtype=np.complex128).reshape(nrec, 6, nf)
    vv = np.ascontiguousarray(np.stack([v.real, v.imag], axis=-1), dtype=np.float64)
    P = _Problem()
    P.n = (C.c_int * 3)(*n)
    P.x = (C.POINTER(C.c_double) * 3)(*[_dp(a) for a in xs])
    P.rd, P.nb, P.ne = rd, nb, ne
    P.sigma = _dp(sigma)
    P.omega0, P.sigma_min, P.dt = omega0, sigma_min, dt
    P.nt, P.fmax = int(nt), fmax
    P.src = (C.c_double * 3)(*[float(a) for a in src])
    P.az, P.dip, P.moment = az, dip, moment
    P.nrec = nrec
    P.rec = _dp(rec) if nrec else None
    P.nfreq = nf
    P.freqs = _dp(freqs) if nf else None
    P.inject, P.pml = int(inject), int(pml)
    grad = np.zeros((3, n[2], n[1], n[0]))
    code = lib.orc_vjp(C.byref(P), _dp(vv), _dp(grad), int(ckpt_every))
    _check(code, "vjp")
    return grad


def forward_workload(w, **kw) -> Dict[str, object]:
    """``forward`` on a :class:`paper_2304_00233_b300.workloads.Workload`-like
    object (duck-typed: only its array attributes are read)."""
    nt = kw.pop("nt", None)
    if nt is None:
        nt = w.nt
    args = dict(rd=w.rd, nb=w.nb, ne=w.ne, omega0=w.omega0, fmax=w.fmax,
                src=w.src, az=w.src_az, dip=w.src_dip, moment=w.moment, rec=w.rec,
                freqs=w.freqs, volume=w.volume)
    args.update(kw)
    if nt is None:
        # one short call to learn dt, then the full run with ceil(t_max/dt) steps
        probe = forward(w.x, w.y, w.z, w.sigma, nt=0, **{**args, "volume": False, "rec": None})
        nt = int(np.ceil(w.t_max / probe["dt"]))
    return forward(w.x, w.y, w.z, w.sigma, nt=nt, **args)


def air_extrapolate(plane, dx: float, dy: float, heights, kind: int) -> np.ndarray:
    """The oracle's air extrapolation of one interface plane [ny][nx] (the top
    boundary of Sec. 3.3): kind 0 gives the same component at each height
    above the interface, [nh][ny][nx]; kind 1 takes H_z and gives H_x, H_y
    at their own x-y positions, [nh][2][ny][nx]."""
    lib = _load()
    plane = _f64(plane)
    ny, nx = plane.shape
    h = _f64(heights)
    nh = len(h)
    out = np.zeros((nh, 2, ny, nx) if kind == 1 else (nh, ny, nx))
    fn = lib.orc_air_extrapolate
    fn.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.POINTER(C.c_double), C.c_int,
                   C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_double)]
    fn.restype = C.c_int
    _check(fn(nx, ny, dx, dy, _dp(plane), nh, _dp(h), int(kind), _dp(out)), "air_extrapolate")
    return out



def _axes(x, y, z):
    xs = [_f64(x), _f64(y), _f64(z)]
    n = (C.c_int * 3)(*[len(a) for a in xs])
    return xs, n, (C.POINTER(C.c_double) * 3)(*[_dp(a) for a in xs])


def stagger(x, y, z, sigma_h, sigma_v) -> np.ndarray:
    """Staggered conductivity [3][n3][n2][n1] from cell values sigma_h,
    sigma_v [n3-1][n2-1][n1-1]: at each E_c sample the mean over the cells
    around its edge weighted by their face areas across it (Sec. 3.6)."""
    xs, n, px = _axes(x, y, z)
    shape = (len(xs[2]) - 1, len(xs[1]) - 1, len(xs[0]) - 1)
    sh, sv = _f64(sigma_h), _f64(sigma_v)
    assert sh.shape == shape and sv.shape == shape, (sh.shape, shape)
    out = np.zeros((3, len(xs[2]), len(xs[1]), len(xs[0])))
    _check(_load().orc_stagger(n, px, _dp(sh), _dp(sv), _dp(out)), "stagger")
    return out


def stagger_T(x, y, z, g):
    """Transpose of :func:`stagger`: (grad_h, grad_v) of a gradient ``g``
    [3][n3][n2][n1] with respect to the staggered conductivity."""
    xs, n, px = _axes(x, y, z)
    g = _f64(g)
    assert g.shape == (3, len(xs[2]), len(xs[1]), len(xs[0])), g.shape
    shape = (len(xs[2]) - 1, len(xs[1]) - 1, len(xs[0]) - 1)
    gh, gv = np.zeros(shape), np.zeros(shape)
    _check(_load().orc_stagger_T(n, px, _dp(g), _dp(gh), _dp(gv)), "stagger_T")
    return gh, gv


def misfit_gradient(x, y, z, sigma_h, sigma_v, d_obs, weight=None, **kw):
    """Least-squares misfit L = 1/2 sum w |G - d_obs|^2 of one transmitter's
    receiver data and its gradient with respect to the cell conductivities:
    G from ``forward`` on ``stagger(sigma_h, sigma_v)``, the cotangent
    w (G - d_obs) through ``vjp`` and then ``stagger_T``.  ``kw`` are the
    arguments ``forward`` and ``vjp`` share (nt, rd, nb, ne, omega0, fmax,
    sigma_min, src, rec, freqs, ...).  Returns dict(misfit, G, grad, grad_h,
    grad_v), grad the staggered-conductivity gradient."""
    sigma = stagger(x, y, z, sigma_h, sigma_v)
    fkw = {k: v for k, v in kw.items() if k != "ckpt_every"}
    G = forward(x, y, z, sigma, **fkw)["G"]
    d = np.asarray(d_obs, dtype=np.complex128).reshape(G.shape)
    w = np.ones(G.shape) if weight is None else np.asarray(weight, dtype=np.float64).reshape(G.shape)
    r = G - d
    misfit = 0.5 * float(np.sum(w * (r.real ** 2 + r.imag ** 2)))
    grad = vjp(x, y, z, sigma, w * r, **kw)
    gh, gv = stagger_T(x, y, z, grad)
    return dict(misfit=misfit, G=G, grad=grad, grad_h=gh, grad_v=gv)
