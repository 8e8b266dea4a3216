"""ctypes wrapper around the C oracle (``rddmc_oracle.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Functions mirror the C
entry points; arrays are numpy.  Unit conversions the C code does not do
(velocity in km/s -> Doppler units with v_th = 12.85 (T/1e4 K)^(1/2) km/s,
Sec. 2.1) happen in the C code.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None


class OrcGrid(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int32), ("n", ctypes.c_int32 * 3), ("J", ctypes.c_int32), ("hybrid", ctypes.c_int32),
        ("R", ctypes.c_double), ("tau0", ctypes.c_double), ("T", ctypes.c_double),
        ("tau_ddmc", ctypes.c_double), ("lam", ctypes.c_double), ("f_mu", ctypes.c_double),
        ("edges", ctypes.c_void_p), ("n_rel", ctypes.c_void_p), ("v", ctypes.c_void_p), ("mask", ctypes.c_void_p),
        ("dust_abs", ctypes.c_double), ("dust_scat", ctypes.c_double), ("redist", ctypes.c_void_p),
        ("dust_weights", ctypes.c_int32), ("pad", ctypes.c_int32),
    ]


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        d, u32, u64, i32, vp = ctypes.c_double, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p
        for name in ("orc_dawson",):
            getattr(L, name).restype = d
            getattr(L, name).argtypes = [d]
        for name in ("orc_voigt_H", "orc_voigt_Hint"):
            getattr(L, name).restype = d
            getattr(L, name).argtypes = [d, d]
        L.orc_bin_mean_H.restype = d
        L.orc_bin_mean_H.argtypes = [d, d, d]
        L.orc_damping.restype = d
        L.orc_damping.argtypes = [d]
        L.orc_philox4x32_10.restype = None
        L.orc_philox4x32_10.argtypes = [vp, vp, vp]
        L.orc_build_table.restype = i32
        L.orc_build_table.argtypes = [ctypes.POINTER(OrcGrid), vp, vp, vp, vp, vp, vp, vp]
        L.orc_tally_len.restype = i32
        L.orc_tally_len.argtypes = [i32]
        L.orc_walk_ddmc.restype = i32
        L.orc_walk_weights.restype = i32
        L.orc_walk_weights.argtypes = [ctypes.POINTER(OrcGrid), vp, vp, vp, vp, vp, d, u64, u64, u64, u64, i32,
                                       vp, vp]
        L.orc_walk_ddmc.argtypes = [ctypes.POINTER(OrcGrid), vp, vp, vp, vp, vp, vp, d, u64, u64, u64, u64, i32, i32,
                                    vp]
        L.orc_walk_slice.restype = i32
        L.orc_walk_slice.argtypes = [ctypes.POINTER(OrcGrid), vp, vp, vp, vp, vp, d, u64, u64, u64, u64, i32, vp]
        L.orc_replay_packet.restype = i32
        L.orc_replay_packet.argtypes = [ctypes.POINTER(OrcGrid), vp, vp, vp, vp, vp, d, u64, u64, u64, u64, vp, vp]
        L.orc_scatter_samples.restype = None
        L.orc_scatter_samples.argtypes = [d, d, u64, u64, vp]
        L.orc_walk_time.restype = ctypes.c_int
        L.orc_walk_time.argtypes = [vp, vp, vp, vp, vp, vp, d, u64, u64, u64, vp, i32, u64, i32, vp, vp, vp, vp, vp,
                                    vp, vp, vp, vp]
        L.orc_fp_samples.restype = None
        L.orc_fp_samples.argtypes = [vp, i32, i32, i32, vp, vp, u64, u64, u64, u64, vp, vp]
        L.orc_fp_region_samples.restype = None
        L.orc_fp_region_samples.argtypes = [ctypes.POINTER(OrcGrid), vp, vp, vp, vp, i32, i32, i32, i32, vp, i32, vp,
                                            vp, u64, u64, u64, u64, vp, vp]
        L.orc_upar_table.restype = None
        L.orc_upar_table.argtypes = [d, vp]
        _LIB = L
    return _LIB


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------- physics
def damping(T: float) -> float:
    return lib().orc_damping(float(T))


def dawson(x):
    f = lib().orc_dawson
    return np.vectorize(lambda v: f(float(v)), otypes=[np.float64])(x)


def voigt_H(a, x):
    f = lib().orc_voigt_H
    return np.vectorize(lambda v: f(float(a), float(v)), otypes=[np.float64])(x)


def voigt_Hint(a, x):
    f = lib().orc_voigt_Hint
    return np.vectorize(lambda v: f(float(a), float(v)), otypes=[np.float64])(x)


def bin_mean_H(a, xlo, xhi):
    f = lib().orc_bin_mean_H
    return np.vectorize(lambda l, h: f(float(a), float(l), float(h)), otypes=[np.float64])(xlo, xhi)


def philox(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


# --------------------------------------------------------------------------- grid / table
def vth_kms(T: float) -> float:
    """Thermal velocity v_th = 12.85 (T/1e4 K)^(1/2) km/s (Sec. 2.1)."""
    return 12.85 * np.sqrt(T / 1.0e4)


class Grid:
    """An oracle grid built from a workload; keeps the numpy buffers alive."""

    def __init__(self, w, hybrid=False, tau_ddmc=5.0, lam=0.7104, f_mu=0.5, n_rel=None, edges=None, dust_abs=0.0,
                 dust_scat=0.0, redist=None, dust_weights=False):
        self.w = w
        e = w.edges() if edges is None else edges
        self.edges = np.ascontiguousarray(e, dtype=np.float64)
        self.n_rel = None if n_rel is None else np.ascontiguousarray(n_rel, dtype=np.float64)
        v = w.velocity_kms()
        self.v = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
        m = w.mask()
        self.mask = None if m is None else np.ascontiguousarray(m, dtype=np.uint8)
        g = OrcGrid()
        g.ndim = w.ndim
        for a in range(3):
            g.n[a] = w.n[a]
        g.J, g.hybrid = w.J, int(hybrid)
        g.R, g.tau0, g.T = w.R, w.tau0, w.T
        g.tau_ddmc, g.lam, g.f_mu = tau_ddmc, lam, f_mu
        g.edges, g.n_rel, g.v, g.mask = (_ptr(self.edges), _ptr(self.n_rel), _ptr(self.v), _ptr(self.mask))
        g.dust_abs, g.dust_scat = float(dust_abs), float(dust_scat)  # grey dust k R at unit density (Sec. 2.6)
        # frequency-grouped MC (Sec. 5.3): J x (J-1) thresholds of eq. R_discrete, kept alive with the grid
        self.redist = None if redist is None else np.ascontiguousarray(redist, dtype=np.uint32)
        g.redist = _ptr(self.redist)
        g.dust_weights = 1 if dust_weights else 0  # continuous absorption by packet weights (Sec. 2.6)
        self.g = g
        self.K = 2 + 2 * w.ndim
        self.KT = self.K + (1 if dust_abs > 0.0 and not dust_weights else 0)  # outcomes, dust absorption last
        self.ncell = w.ncell
        self.J = w.J

    def table(self):
        nS = self.ncell * self.J
        K = self.KT  # with dust absorption one more outcome (the last)
        t = dict(
            thr=np.zeros(nS * (K - 1), dtype=np.uint32), flags=np.zeros(nS, dtype=np.uint32),
            rebin_m=np.zeros(self.ncell * 2 * self.w.ndim, dtype=np.int32),
            rebin_thr=np.zeros(self.ncell * 2 * self.w.ndim, dtype=np.uint32),
            k=np.zeros(nS, dtype=np.float64), rate=np.zeros(nS * K, dtype=np.float64),
            surv=np.zeros(nS, dtype=np.float64))
        rc = lib().orc_build_table(ctypes.byref(self.g), _ptr(t["thr"]), _ptr(t["flags"]), _ptr(t["rebin_m"]),
                                   _ptr(t["rebin_thr"]), _ptr(t["k"]), _ptr(t["rate"]), _ptr(t["surv"]))
        if rc != 0:
            raise RuntimeError(f"orc_build_table failed: {rc}")
        t["thr"] = t["thr"].reshape(nS, K - 1)
        t["rate"] = t["rate"].reshape(nS, K)
        return t


NSB = 64          # impact-parameter bins over b/R in [0, 1.28)
SB_MAX = 1.28
TALLY_NAMES = ["emitted", "escaped", "aborted", "steps", "mc_events", "conversions", "clamps", "event_draws",
               "absorbed"]
_T_FACE, _T_HIST = 9, 15


def unpack_tally(t: np.ndarray, J: int) -> dict:
    d = {name: int(t[i]) for i, name in enumerate(TALLY_NAMES)}
    d["faces"] = t[_T_FACE:_T_FACE + 6].astype(np.uint64).copy()
    d["hist"] = t[_T_HIST:_T_HIST + J + 2].astype(np.uint64).copy()
    d["sb"] = t[_T_HIST + J + 2:_T_HIST + J + 2 + NSB].astype(np.uint64).copy()
    return d


def walk_weights(grid: Grid, table: dict, seed: int, p0: int, npk: int, max_steps: int = (1 << 62),
                 nthreads: int = 0) -> dict:
    """The DDMC walk with continuous absorption by packet weights (orc_walk_weights;
    a grid with dust_weights): the integer tallies plus the escaped weight, in
    total (escaped_weight) and per escape-histogram bin (weight_hist, J + 2)."""
    if nthreads <= 0:
        nthreads = os.cpu_count() or 1
    out = np.zeros(lib().orc_tally_len(grid.J), dtype=np.uint64)
    wt = np.zeros(grid.J + 3, dtype=np.float64)
    thr = np.ascontiguousarray(table["thr"].ravel())
    rc = lib().orc_walk_weights(ctypes.byref(grid.g), _ptr(thr), _ptr(table["flags"]), _ptr(table["rebin_m"]),
                                _ptr(table["rebin_thr"]), _ptr(table["surv"]), float(grid.w.x0), int(seed), int(p0),
                                int(npk), int(max_steps), int(nthreads), _ptr(out), _ptr(wt))
    if rc != 0:
        raise RuntimeError(f"orc_walk_weights failed: {rc}")
    d = unpack_tally(out, grid.J)
    d.update(escaped_weight=float(wt[0]), weight_hist=wt[1:].copy())
    return d


def walk(grid: Grid, table: dict, seed: int, p0: int, npk: int, max_steps: int = (1 << 62),
         literal: bool = False, nthreads: int = 0) -> dict:
    """Run packets [p0, p0+npk) of the DDMC walk; returns the integer tallies."""
    if nthreads <= 0:
        nthreads = os.cpu_count() or 1
    L = lib().orc_tally_len(grid.J)
    out = np.zeros(L, dtype=np.uint64)
    thr = np.ascontiguousarray(table["thr"].ravel())
    rate = np.ascontiguousarray(table["rate"].ravel())
    rc = lib().orc_walk_ddmc(ctypes.byref(grid.g), _ptr(thr), _ptr(table["flags"]), _ptr(table["rebin_m"]),
                             _ptr(table["rebin_thr"]), _ptr(rate), _ptr(table["k"]), float(grid.w.x0), int(seed), int(p0),
                             int(npk), int(max_steps), int(literal), int(nthreads), _ptr(out))
    if rc == -1:
        raise ValueError("orc_walk_ddmc: bad input")
    res = unpack_tally(out, grid.J)
    res["status"] = rc
    return res


def replay_packet(grid: Grid, table: dict, seed: int, pid: int, n_trans: int, max_steps: int = (1 << 62)) -> dict:
    """State of one packet after at most n_trans transitions (the oracle's own table)."""
    out = np.zeros(5, dtype=np.uint64)
    tl = np.zeros(lib().orc_tally_len(grid.J), dtype=np.uint64)
    thr = np.ascontiguousarray(table["thr"].ravel())
    rc = lib().orc_replay_packet(ctypes.byref(grid.g), _ptr(thr), _ptr(table["flags"]), _ptr(table["rebin_m"]),
                                 _ptr(table["rebin_thr"]), _ptr(table["k"]), float(grid.w.x0), int(seed), int(pid),
                                 int(n_trans),
                                 int(max_steps), _ptr(out), _ptr(tl))
    if rc == -1:
        raise ValueError("orc_replay_packet: bad input")
    d = dict(cell=int(out[0]), bin=int(out[1]), steps=int(out[2]), event_draws=int(out[3]), done=int(out[4]))
    d["tally"] = unpack_tally(tl, grid.J)
    return d


def walk_time(grid: Grid, table: dict, seed: int, p0: int, npk: int, t_edges, max_steps: int = (1 << 62),
              nthreads: int = 0, leaks: bool = False) -> dict:
    """Time-dependent walk of packets [p0, p0+npk) emitted at t_edges[0]
    (orc_walk_time): per step n the packets in each state at its end (bins,
    nt x S), the path length spent in each state (path, nt x S) and the
    escapes (esc, nt), plus the walk's tallies and transition/dwell counts.
    leaks=True adds the optical depths of the leaks of eq. a_estimator
    (leak, nt x ncell x 2 ndim x 2: per face, leaving / entering the cell)."""
    if nthreads <= 0:
        nthreads = os.cpu_count() or 1
    te = np.ascontiguousarray(t_edges, dtype=np.float64)
    nt = len(te) - 1
    S = grid.ncell * grid.J
    nf = 2 * grid.w.ndim
    bins = np.zeros(nt * S, dtype=np.uint64)
    path = np.zeros(nt * S, dtype=np.float64)
    esc = np.zeros(nt, dtype=np.uint64)
    tally = np.zeros(lib().orc_tally_len(grid.J), dtype=np.uint64)
    stats = np.zeros(3, dtype=np.uint64)
    leak = np.zeros(nt * grid.ncell * nf * 2, dtype=np.float64) if leaks else None
    weighted = bool(grid.g.dust_weights)
    wbins = np.zeros(nt * S, dtype=np.float64) if weighted else None
    wpath = np.zeros(nt * S, dtype=np.float64) if weighted else None
    thr = np.ascontiguousarray(table["thr"].ravel())
    rate = np.ascontiguousarray(table["rate"].ravel())
    rc = lib().orc_walk_time(ctypes.byref(grid.g), _ptr(thr), _ptr(table["flags"]), _ptr(table["rebin_m"]),
                             _ptr(table["rebin_thr"]), _ptr(rate), float(grid.w.x0), int(seed), int(p0), int(npk),
                             _ptr(te), int(nt), int(max_steps), int(nthreads), _ptr(bins), _ptr(path), _ptr(esc),
                             _ptr(tally), _ptr(stats), _ptr(table["k"]) if leaks else None, _ptr(leak), _ptr(wbins),
                             _ptr(wpath))
    if rc != 0:
        raise RuntimeError(f"orc_walk_time failed: {rc}")
    out = unpack_tally(tally, grid.J)
    out.update(bins=bins.reshape(nt, S), path=path.reshape(nt, S), esc=esc, transitions=int(stats[0]),
               dwells=int(stats[1]), aborted_time=int(stats[2]))
    if leaks:
        out["leak"] = leak.reshape(nt, grid.ncell, nf, 2)
    if weighted:  # dust by packet weights: weighted bin and path estimates
        out["wbins"] = wbins.reshape(nt, S)
        out["wpath"] = wpath.reshape(nt, S)
    return out


def walk_slice(grid: Grid, table: dict, seed: int, p0: int, npk: int, n_trans: int, nthreads: int = 0) -> dict:
    """Start packets [p0, p0+npk) and advance each by at most n_trans transitions."""
    if nthreads <= 0:
        nthreads = os.cpu_count() or 1
    out = np.zeros(lib().orc_tally_len(grid.J), dtype=np.uint64)
    thr = np.ascontiguousarray(table["thr"].ravel())
    rc = lib().orc_walk_slice(ctypes.byref(grid.g), _ptr(thr), _ptr(table["flags"]), _ptr(table["rebin_m"]),
                              _ptr(table["rebin_thr"]), _ptr(table["k"]), float(grid.w.x0), int(seed), int(p0),
                              int(npk),
                              int(n_trans), int(nthreads), _ptr(out))
    if rc == -1:
        raise ValueError("orc_walk_slice: bad input")
    res = unpack_tally(out, grid.J)
    res["status"] = rc
    return res


def scatter_samples(T: float, x_in: float, seed: int, n: int) -> np.ndarray:
    """Outgoing frequencies of n independent scatterings at x_in (density R_II-A)."""
    out = np.zeros(n, dtype=np.float64)
    lib().orc_scatter_samples(float(T), float(x_in), int(seed), int(n), _ptr(out))
    return out


def upar_table(T: float) -> np.ndarray:
    """Envelope split points (u1, u0) of the u_par sampler on the |x| grid (step 1/16)."""
    out = np.zeros(2 * 1024, dtype=np.float64)
    lib().orc_upar_table(float(damping(T)), _ptr(out))
    return out.reshape(1024, 2)


def interior_rows(w_uniform) -> np.ndarray:
    """Rows (7 thresholds + flags per bin) of an interior cell of a uniform 3D
    medium: the centre cell of a 3^3 grid of the workload's density."""
    w3 = w_uniform.with_(n=(3, 3, 3), ndim=3, sphere=False, vmax_kms=0.0)
    g = Grid(w3)
    t = g.table()
    c = 13  # centre cell of 3^3
    thr = t["thr"].reshape(27, w3.J, 7)[c]
    fl = t["flags"].reshape(27, w3.J)[c]
    return np.concatenate([thr, fl[:, None]], axis=1).astype(np.uint32)


def fp_samples(rows: np.ndarray, b: int, jlo, jhi, seed: int, p0: int, n: int, cap: int):
    """First passages through a uniform brick (see orc_fp_samples): records
    [n x 8] {level, start bin, folded start cell, exit face, exit bin, exit
    position, 0, 0} and transition counts."""
    rows = np.ascontiguousarray(rows, dtype=np.uint32)
    L, J = rows.shape[0], rows.shape[1]
    jlo = np.ascontiguousarray(jlo, dtype=np.int32)
    jhi = np.ascontiguousarray(jhi, dtype=np.int32)
    out = np.zeros(8 * n, dtype=np.int32)
    steps = np.zeros(n, dtype=np.uint64)
    lib().orc_fp_samples(_ptr(rows), int(L), int(J), int(b), _ptr(jlo), _ptr(jhi), int(seed), int(p0), int(n),
                         int(cap), _ptr(out), _ptr(steps))
    return out.reshape(n, 8), steps


def fp_region_samples(grid: Grid, table: dict, bl: int, sh: int, m: int, nbx: int, bricks, off, bins, seed: int,
                      p0: int, n: int, cap: int):
    """First passages out of the regions (inner cubes) of bricks of the grid's
    own medium (see orc_fp_region_samples): records [n x 8] {brick, start bin,
    start cell, exit face, exit bin, exit cell on the face, rebin draws, 0} and
    transition counts."""
    bricks = np.ascontiguousarray(bricks, dtype=np.int32)
    off = np.ascontiguousarray(off, dtype=np.int32)
    bins = np.ascontiguousarray(bins, dtype=np.int32)
    out = np.zeros(8 * n, dtype=np.int32)
    steps = np.zeros(n, dtype=np.uint64)
    thr = np.ascontiguousarray(table["thr"].ravel())
    lib().orc_fp_region_samples(ctypes.byref(grid.g), _ptr(thr), _ptr(table["flags"]), _ptr(table["rebin_m"]),
                                _ptr(table["rebin_thr"]), int(bl), int(sh), int(m), int(nbx), _ptr(bricks),
                                int(len(bricks)), _ptr(off), _ptr(bins), int(seed), int(p0), int(n), int(cap),
                                _ptr(out), _ptr(steps))
    return out.reshape(n, 8), steps
