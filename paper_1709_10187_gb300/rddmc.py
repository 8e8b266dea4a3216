"""Thin ctypes binding of the C-ABI in ``include/rddmc.h``.

Argument marshalling only: every step of the walk runs in the CUDA library.
PyTorch supplies device memory (tensors whose ``data_ptr()`` is passed) and
streams.  Loading fails loudly when the library has not been built; there is no
CPU fallback.

Low-level functions mirror the C names (``build_grid``, ``grid_sizes``,
``precompute_leakage``, ``reset_tallies``, ``launch_packets``,
``read_tallies``, ``table_rows``).  ``Problem`` bundles them for a workload:
it owns the handle and the caller-side device buffers.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "librddmc.so")

OK, ERR_ARG, ERR_UNSUPPORTED, ERR_SIZE, ERR_CUDA, ERR_STEP_LIMIT, ERR_TABLE, ERR_TIMEOUT = 0, -1, -2, -3, -4, -5, -6, -7
GEOM_SLAB_1D, GEOM_CART_3D = 1, 3
MODE_DDMC, MODE_HYBRID = 0, 1
LAYOUT_DEDUP, LAYOUT_DENSE = 0, 1
DUST_PROBABILISTIC, DUST_WEIGHTS = 0, 1
NSB = 64  # impact-parameter bins of the surface-brightness histogram

EXPORTED = ["rddmc_build_grid", "rddmc_destroy_grid", "rddmc_grid_sizes", "rddmc_precompute_leakage",
            "rddmc_reset_tallies", "rddmc_launch_packets", "rddmc_read_tallies", "rddmc_table_rows",
            "rddmc_read_packet_states", "rddmc_launch_packets_noalloc", "rddmc_gather_probe", "rddmc_scatter_samples",
            "rddmc_batch_create", "rddmc_batch_destroy", "rddmc_batch_sizes", "rddmc_batch_upload",
            "rddmc_batch_launch", "rddmc_batch_read_tallies", "rddmc_batch_graph_create", "rddmc_batch_graph_launch",
            "rddmc_batch_graph_destroy", "rddmc_batch_autotune", "rddmc_cell_tau", "rddmc_fp_generate",
            "rddmc_fp_region_generate",
            "rddmc_mlp_param_count", "rddmc_mlp_work_bytes", "rddmc_mlp_to_bf16", "rddmc_mlp_forward",
            "rddmc_mlp_loss_grad", "rddmc_mlp_adam", "rddmc_mlp_status", "rddmc_propose", "rddmc_time_state_bytes",
            "rddmc_time_step_launch", "rddmc_redistribution_bytes", "rddmc_precompute_redistribution",
            "rddmc_read_escape_weights",
            "rddmc_status_string", "rddmc_version"]

TIME_TICKS = 1 << 31  # ticks per time step in the path tallies of rddmc_time_step_launch


class GridDesc(ctypes.Structure):
    _fields_ = [("geometry", ctypes.c_int32), ("n", ctypes.c_int32 * 3), ("nbins", ctypes.c_int32),
                ("layout", ctypes.c_int32), ("R", ctypes.c_double), ("tau0", ctypes.c_double),
                ("T", ctypes.c_double), ("freq_edges", ctypes.c_void_p), ("n_rel", ctypes.c_void_p),
                ("v_kms", ctypes.c_void_p), ("mask", ctypes.c_void_p)]


class LeakParams(ctypes.Structure):
    _fields_ = [("tau_ddmc", ctypes.c_double), ("lam", ctypes.c_double), ("f_mu", ctypes.c_double),
                ("mode", ctypes.c_int32), ("dust_method", ctypes.c_int32), ("dust_abs", ctypes.c_double),
                ("dust_scat", ctypes.c_double)]


class RunOpts(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("n_packets", ctypes.c_uint64), ("max_steps", ctypes.c_uint64),
                ("steps_per_launch", ctypes.c_uint64), ("resume", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("threads_per_cta", ctypes.c_int32), ("chunk", ctypes.c_int32), ("table_in_smem", ctypes.c_int32),
                ("time_slice_us", ctypes.c_int32), ("proposal", ctypes.c_void_p), ("redist", ctypes.c_void_p)]


class Sizes(ctypes.Structure):
    _fields_ = [("table_bytes", ctypes.c_uint64), ("tally_bytes", ctypes.c_uint64), ("state_bytes", ctypes.c_uint64),
                ("n_class", ctypes.c_int32), ("row_bytes", ctypes.c_int32), ("n_outcomes", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class Tallies(ctypes.Structure):
    _fields_ = [("emitted", ctypes.c_uint64), ("escaped", ctypes.c_uint64), ("aborted", ctypes.c_uint64),
                ("steps", ctypes.c_uint64), ("mc_events", ctypes.c_uint64), ("conversions", ctypes.c_uint64),
                ("clamps", ctypes.c_uint64), ("event_draws", ctypes.c_uint64), ("proposals", ctypes.c_uint64),
                ("proposed_steps", ctypes.c_uint64), ("absorbed", ctypes.c_uint64),
                ("escaped_weight", ctypes.c_double), ("status", ctypes.c_int32),
                ("nbins", ctypes.c_int32), ("nfaces", ctypes.c_int32), ("nsb", ctypes.c_int32)]


class FpTrain(ctypes.Structure):
    _fields_ = [("d_x", ctypes.c_void_p), ("d_ta", ctypes.c_void_p), ("d_tb", ctypes.c_void_p),
                ("d_lk", ctypes.c_void_p), ("d_lp", ctypes.c_void_p), ("d_xc", ctypes.c_void_p),
                ("d_tc", ctypes.c_void_p)]


class Proposal(ctypes.Structure):
    _fields_ = [("brick", ctypes.c_int32), ("offset", ctypes.c_int32), ("d_brick_lk", ctypes.c_void_p),
                ("d_lp", ctypes.c_void_p), ("d_xc", ctypes.c_void_p), ("log_tau_lo", ctypes.c_double),
                ("log_tau_hi", ctypes.c_double), ("d_queue_count", ctypes.c_void_p), ("d_queue_pid", ctypes.c_void_p),
                ("n_bricks", ctypes.c_int32), ("margin", ctypes.c_int32), ("d_summary", ctypes.c_void_p)]


class FpRegion(ctypes.Structure):
    _fields_ = [("brick", ctypes.c_int32), ("offset", ctypes.c_int32), ("margin", ctypes.c_int32),
                ("n_eligible", ctypes.c_int32), ("d_bricks", ctypes.c_void_p), ("d_bin_off", ctypes.c_void_p),
                ("d_bins", ctypes.c_void_p), ("d_summary", ctypes.c_void_p)]


class TimeStep(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("n_packets", ctypes.c_uint64), ("max_steps", ctypes.c_uint64),
                ("t_begin", ctypes.c_double), ("t_end", ctypes.c_double), ("start", ctypes.c_int32),
                ("chunk", ctypes.c_int32), ("threads_per_cta", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("regroup", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class RDDMCError(RuntimeError):
    def __init__(self, fn: str, status: int):
        super().__init__(f"{fn} failed: {status} ({status_string(status)})")
        self.status = status


_LIB = None


def lib():
    """Load the CUDA library; raises if it has not been built (no fallback)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run paper_1709_10187_gb300.build.build())")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, u64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_size_t
        L.rddmc_build_grid.argtypes = [ctypes.POINTER(GridDesc), ctypes.POINTER(vp)]
        L.rddmc_destroy_grid.argtypes = [vp]
        L.rddmc_destroy_grid.restype = None
        L.rddmc_grid_sizes.argtypes = [vp, u64, ctypes.POINTER(Sizes)]
        L.rddmc_precompute_leakage.argtypes = [vp, ctypes.POINTER(LeakParams), vp, sz, vp]
        L.rddmc_reset_tallies.argtypes = [vp, vp, sz, vp]
        L.rddmc_launch_packets.argtypes = [vp, vp, ctypes.POINTER(RunOpts), vp, sz, vp, sz, vp]
        L.rddmc_read_tallies.argtypes = [vp, vp, ctypes.POINTER(Tallies), vp, vp, vp, vp]
        L.rddmc_table_rows.argtypes = [vp, vp, vp, vp, vp]
        L.rddmc_read_packet_states.argtypes = [vp, vp, u64, u64, u64, vp, vp, vp, vp, vp, vp]
        L.rddmc_launch_packets_noalloc.argtypes = [vp, vp, ctypes.POINTER(RunOpts), vp, sz, vp]
        L.rddmc_gather_probe.argtypes = [vp, u64, i32, i32, ctypes.c_uint32, i32, i32, u64, i32, vp,
                                         ctypes.POINTER(u64), vp]
        L.rddmc_scatter_samples.argtypes = [vp, vp, ctypes.c_double, u64, u64, vp, vp]
        L.rddmc_cell_tau.argtypes = [vp, vp, ctypes.c_int64, vp, vp]
        L.rddmc_fp_generate.argtypes = [vp, vp, i32, i32, vp, vp, u64, u64, u64, u64, vp, vp,
                                        ctypes.POINTER(FpTrain), vp]
        L.rddmc_fp_region_generate.argtypes = [vp, vp, ctypes.POINTER(FpRegion), u64, u64, u64, u64, vp, vp,
                                                ctypes.POINTER(FpTrain), vp]
        L.rddmc_propose.argtypes = [vp, vp, ctypes.POINTER(Proposal), u64, u64, vp, vp, i32, i32, i32, i32, vp, vp, i32,
                                    vp, ctypes.POINTER(ctypes.c_uint64), vp]
        L.rddmc_mlp_param_count.argtypes = [i32]
        L.rddmc_mlp_status.argtypes = [vp]
        L.rddmc_mlp_work_bytes.argtypes = [i32, i32]
        L.rddmc_mlp_to_bf16.argtypes = [i32, vp, vp, vp]
        L.rddmc_mlp_forward.argtypes = [i32, vp, vp, vp, i32, vp, vp, vp]
        L.rddmc_mlp_loss_grad.argtypes = [i32, i32, i32, i32, i32, vp, vp, vp, vp, vp, vp, i32, vp, vp, vp, vp]
        L.rddmc_mlp_adam.argtypes = [i32, vp, vp, vp, vp, vp, i32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                     ctypes.c_float, vp]
        L.rddmc_batch_create.argtypes = [vp, vp, vp, i32, ctypes.POINTER(vp)]
        L.rddmc_batch_destroy.argtypes = [vp]
        L.rddmc_batch_destroy.restype = None
        L.rddmc_batch_sizes.argtypes = [vp, vp, vp, vp, vp]
        L.rddmc_batch_upload.argtypes = [vp, ctypes.c_double, vp, sz, vp]
        L.rddmc_batch_launch.argtypes = [vp, vp, ctypes.POINTER(RunOpts), i32, vp, sz, vp, sz, vp]
        L.rddmc_batch_read_tallies.argtypes = [vp, vp, i32, ctypes.POINTER(Tallies), vp, vp, vp, vp]
        L.rddmc_batch_graph_create.argtypes = [vp, vp, ctypes.POINTER(RunOpts), vp, sz, vp, sz, vp, ctypes.POINTER(vp)]
        L.rddmc_batch_graph_launch.argtypes = [vp, vp]
        L.rddmc_batch_graph_destroy.argtypes = [vp]
        L.rddmc_batch_graph_destroy.restype = None
        L.rddmc_batch_autotune.argtypes = [vp, vp, ctypes.POINTER(RunOpts), vp, sz, vp, sz, vp, ctypes.POINTER(RunOpts),
                                           ctypes.POINTER(ctypes.c_double)]
        L.rddmc_time_state_bytes.argtypes = [u64]
        L.rddmc_redistribution_bytes.argtypes = [vp]
        L.rddmc_read_escape_weights.argtypes = [vp, vp, vp, vp]
        L.rddmc_precompute_redistribution.argtypes = [vp, vp, i32, vp, sz, vp]
        L.rddmc_time_step_launch.argtypes = [vp, vp, ctypes.POINTER(TimeStep), vp, sz, vp, sz, vp, vp, vp, vp, vp, vp,
                                             vp]
        L.rddmc_status_string.argtypes = [i32]
        L.rddmc_status_string.restype = ctypes.c_char_p
        L.rddmc_version.argtypes = []
        for name in EXPORTED:
            if name not in ("rddmc_destroy_grid", "rddmc_status_string", "rddmc_batch_destroy",
                            "rddmc_batch_graph_destroy"):
                getattr(L, name).restype = ctypes.c_int
        L.rddmc_mlp_param_count.restype = ctypes.c_uint64
        L.rddmc_mlp_work_bytes.restype = ctypes.c_uint64
        L.rddmc_time_state_bytes.restype = ctypes.c_uint64
        L.rddmc_redistribution_bytes.restype = ctypes.c_uint64
        _LIB = L
    return _LIB


def status_string(s: int) -> str:
    return lib().rddmc_status_string(int(s)).decode()


def _check(fn: str, s: int):
    if s != OK:
        raise RDDMCError(fn, s)


def _np_ptr(a: Optional[np.ndarray]):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


# ----------------------------------------------------------------------------- C names
def build_grid(geometry, n, edges, R, tau0, T, n_rel=None, v_kms=None, mask=None, layout=LAYOUT_DEDUP):
    """rddmc_build_grid; returns an opaque handle (int)."""
    e = np.ascontiguousarray(edges, dtype=np.float64)
    nr = None if n_rel is None else np.ascontiguousarray(n_rel, dtype=np.float64)
    v = None if v_kms is None else np.ascontiguousarray(v_kms, dtype=np.float64)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    d = GridDesc()
    d.geometry = geometry
    for a in range(3):
        d.n[a] = int(n[a])
    d.nbins = len(e) - 1
    d.layout = layout
    d.R, d.tau0, d.T = float(R), float(tau0), float(T)
    d.freq_edges, d.n_rel, d.v_kms, d.mask = (ctypes.c_void_p(e.ctypes.data), _np_ptr(nr), _np_ptr(v), _np_ptr(m))
    h = ctypes.c_void_p()
    _check("rddmc_build_grid", lib().rddmc_build_grid(ctypes.byref(d), ctypes.byref(h)))
    return h.value


def destroy_grid(grid):
    if grid:
        lib().rddmc_destroy_grid(ctypes.c_void_p(grid))


def grid_sizes(grid, n_packets: int) -> Sizes:
    s = Sizes()
    _check("rddmc_grid_sizes", lib().rddmc_grid_sizes(ctypes.c_void_p(grid), int(n_packets), ctypes.byref(s)))
    return s


def precompute_leakage(grid, params: LeakParams, d_table: int, table_bytes: int, stream: int = 0):
    _check("rddmc_precompute_leakage", lib().rddmc_precompute_leakage(
        ctypes.c_void_p(grid), ctypes.byref(params), ctypes.c_void_p(d_table), int(table_bytes),
        ctypes.c_void_p(stream)))


def reset_tallies(grid, d_tallies: int, tally_bytes: int, stream: int = 0):
    _check("rddmc_reset_tallies", lib().rddmc_reset_tallies(ctypes.c_void_p(grid), ctypes.c_void_p(d_tallies),
                                                            int(tally_bytes), ctypes.c_void_p(stream)))


def launch_packets(grid, d_table: int, opts: RunOpts, d_state: int, state_bytes: int, d_tallies: int,
                   tally_bytes: int, stream: int = 0):
    _check("rddmc_launch_packets", lib().rddmc_launch_packets(
        ctypes.c_void_p(grid), ctypes.c_void_p(d_table), ctypes.byref(opts), ctypes.c_void_p(d_state),
        int(state_bytes), ctypes.c_void_p(d_tallies), int(tally_bytes), ctypes.c_void_p(stream)))


def launch_packets_noalloc(grid, d_table: int, opts: RunOpts, d_tallies: int, tally_bytes: int, stream: int = 0):
    """rddmc_launch_packets_noalloc: the walk with the library's fixed scratch
    array in place of a caller state buffer (for callers that cannot allocate
    device memory); concurrent calls race on that array."""
    _check("rddmc_launch_packets_noalloc", lib().rddmc_launch_packets_noalloc(
        ctypes.c_void_p(grid), ctypes.c_void_p(d_table), ctypes.byref(opts), ctypes.c_void_p(d_tallies),
        int(tally_bytes), ctypes.c_void_p(stream)))


def gather_probe(d_table: int, table_bytes: int, row_bytes: int, in_smem: bool, chain: int, ctas_per_sm: int,
                 threads_per_cta: int, seed: int, fill: bool, d_sink: int, stream: int = 0) -> int:
    """rddmc_gather_probe: launch the random dependent-gather chase; returns the
    number of loads the launch makes (time it with events on `stream`)."""
    n = ctypes.c_uint64(0)
    _check("rddmc_gather_probe", lib().rddmc_gather_probe(
        ctypes.c_void_p(d_table), int(table_bytes), int(row_bytes), int(bool(in_smem)), int(chain), int(ctas_per_sm),
        int(threads_per_cta), int(seed), int(bool(fill)), ctypes.c_void_p(d_sink), ctypes.byref(n),
        ctypes.c_void_p(stream)))
    return int(n.value)


def redistribution_bytes(grid) -> int:
    """rddmc_redistribution_bytes."""
    return int(lib().rddmc_redistribution_bytes(ctypes.c_void_p(grid)))


def precompute_redistribution(grid, d_table: int, n_sub: int, d_redist: int, nbytes: int, stream: int = 0):
    """rddmc_precompute_redistribution (eq. R_discrete thresholds; enqueued)."""
    _check("rddmc_precompute_redistribution", lib().rddmc_precompute_redistribution(
        ctypes.c_void_p(grid), ctypes.c_void_p(d_table), int(n_sub), ctypes.c_void_p(d_redist), int(nbytes),
        ctypes.c_void_p(stream)))


def time_state_bytes(n_packets: int) -> int:
    """rddmc_time_state_bytes."""
    return int(lib().rddmc_time_state_bytes(int(n_packets)))


def time_step_launch(grid, d_table: int, step: TimeStep, d_state: int, state_bytes: int, d_tallies: int,
                     tally_bytes: int, d_bins: int, d_path: int, d_counts: int, stream: int = 0, d_leak: int = 0,
                     d_wbins: int = 0, d_wpath: int = 0):
    """rddmc_time_step_launch (enqueues one time step; no synchronisation)."""
    _check("rddmc_time_step_launch", lib().rddmc_time_step_launch(
        ctypes.c_void_p(grid), ctypes.c_void_p(d_table), ctypes.byref(step), ctypes.c_void_p(d_state),
        int(state_bytes), ctypes.c_void_p(d_tallies), int(tally_bytes), ctypes.c_void_p(d_bins),
        ctypes.c_void_p(d_path), ctypes.c_void_p(d_counts), ctypes.c_void_p(d_leak or None),
        ctypes.c_void_p(d_wbins or None), ctypes.c_void_p(d_wpath or None), ctypes.c_void_p(stream)))


def scatter_samples(grid, d_table: int, x_in: float, seed: int, n: int, d_out: int, stream: int = 0):
    """rddmc_scatter_samples: n outgoing frequencies of the device scattering sampler."""
    _check("rddmc_scatter_samples", lib().rddmc_scatter_samples(
        ctypes.c_void_p(grid), ctypes.c_void_p(d_table), float(x_in), int(seed), int(n), ctypes.c_void_p(d_out),
        ctypes.c_void_p(stream)))


def read_tallies(grid, d_tallies: int, J: int, nfaces: int, stream: int = 0) -> dict:
    t = Tallies()
    hist = np.zeros(J + 2, dtype=np.uint64)
    faces = np.zeros(nfaces, dtype=np.uint64)
    sb = np.zeros(NSB, dtype=np.uint64)
    _check("rddmc_read_tallies", lib().rddmc_read_tallies(ctypes.c_void_p(grid), ctypes.c_void_p(d_tallies),
                                                          ctypes.byref(t), _np_ptr(hist), _np_ptr(faces),
                                                          _np_ptr(sb), ctypes.c_void_p(stream)))
    d = {k: getattr(t, k) if k == "escaped_weight" else int(getattr(t, k)) for k, _ in Tallies._fields_}
    whist = np.zeros(J + 2, dtype=np.float64)
    _check("rddmc_read_escape_weights", lib().rddmc_read_escape_weights(
        ctypes.c_void_p(grid), ctypes.c_void_p(d_tallies), _np_ptr(whist), ctypes.c_void_p(stream)))
    d["weight_hist"] = whist
    d["hist"] = hist
    d["faces"] = faces
    d["sb"] = sb
    return d


def table_rows(grid, d_table: int, ncell: int, J: int, K: int, stream: int = 0):
    thr = np.zeros(ncell * J * (K - 1), dtype=np.uint32)
    flags = np.zeros(ncell * J, dtype=np.uint32)
    _check("rddmc_table_rows", lib().rddmc_table_rows(ctypes.c_void_p(grid), ctypes.c_void_p(d_table),
                                                      _np_ptr(thr), _np_ptr(flags), ctypes.c_void_p(stream)))
    return thr.reshape(ncell * J, K - 1), flags


def read_packet_states(grid, d_state: int, n_packets: int, first: int, count: int, stream: int = 0) -> dict:
    out = dict(cell=np.zeros(count, np.uint32), bin=np.zeros(count, np.uint32), steps=np.zeros(count, np.uint64),
               event_draws=np.zeros(count, np.uint64), status=np.zeros(count, np.uint8))
    _check("rddmc_read_packet_states", lib().rddmc_read_packet_states(
        ctypes.c_void_p(grid), ctypes.c_void_p(d_state), int(n_packets), int(first), int(count),
        _np_ptr(out["cell"]), _np_ptr(out["bin"]), _np_ptr(out["steps"]), _np_ptr(out["event_draws"]),
        _np_ptr(out["status"]), ctypes.c_void_p(stream)))
    return out


# ----------------------------------------------------------------------------- convenience
class Problem:
    """A workload bound to the library: handle, table, tallies and packet state
    in caller-owned torch device buffers."""

    def __init__(self, w, mode=MODE_DDMC, layout=LAYOUT_DEDUP, tau_ddmc=5.0, lam=0.7104, f_mu=0.5,
                 device="cuda", n_rel=None, edges=None, v_kms=None, dust_abs=0.0, dust_scat=0.0,
                 dust_weights=False):
        import torch
        self.torch = torch
        self.w = w
        self.device = torch.device(device)
        geom = GEOM_SLAB_1D if w.ndim == 1 else GEOM_CART_3D
        self.edges = np.asarray(w.edges() if edges is None else edges, dtype=np.float64)
        self.grid = build_grid(geom, w.n, self.edges, w.R, w.tau0, w.T, n_rel=n_rel,
                               v_kms=w.velocity_kms() if v_kms is None else v_kms, mask=w.mask(), layout=layout)
        self.J = len(self.edges) - 1
        self.nfaces = 2 * w.ndim
        self.K = 2 + 2 * w.ndim
        s = grid_sizes(self.grid, 1)
        self.sizes = s
        self.table = torch.empty(int(s.table_bytes), dtype=torch.uint8, device=self.device)
        self.tally = torch.zeros(int(s.tally_bytes) // 8, dtype=torch.int64, device=self.device)
        self.state = None
        self.state_packets = 0
        self.params = LeakParams(tau_ddmc, lam, f_mu, mode, DUST_WEIGHTS if dust_weights else DUST_PROBABILISTIC,
                                 dust_abs, dust_scat)
        precompute_leakage(self.grid, self.params, self.table.data_ptr(), self.table.numel(), self.stream())

    def stream(self) -> int:
        return self.torch.cuda.current_stream(self.device).cuda_stream

    def ensure_state(self, n_packets: int):
        need = int(grid_sizes(self.grid, n_packets).state_bytes)
        if self.state is None or self.state.numel() < need:
            self.state = self.torch.empty(need, dtype=self.torch.uint8, device=self.device)
        return self.state

    def reset(self):
        reset_tallies(self.grid, self.tally.data_ptr(), self.tally.numel() * 8, self.stream())

    @classmethod
    def clumpy(cls, med, **kw):
        """A Problem on a clumpy medium (workloads.ClumpyMedium): its density and
        turbulent velocity per cell."""
        return cls(med.workload, n_rel=med.n_rel, v_kms=med.v_kms, **kw)

    def launch(self, n_packets: int, seed: int, max_steps: int = 0, steps_per_launch: int = 0, resume: int = 0,
               ctas_per_sm: int = 0, threads_per_cta: int = 0, chunk: int = 0, table_in_smem: int = 0,
               proposal: "Proposal" = None, time_slice_us: int = 0, redist=None):
        st = self.ensure_state(n_packets)
        o = RunOpts(seed, n_packets, max_steps, steps_per_launch, resume, ctas_per_sm, threads_per_cta, chunk,
                    table_in_smem, time_slice_us, ctypes.addressof(proposal) if proposal is not None else None,
                    redist.data_ptr() if redist is not None else None)
        launch_packets(self.grid, self.table.data_ptr(), o, st.data_ptr(), st.numel(), self.tally.data_ptr(),
                       self.tally.numel() * 8, self.stream())

    def read(self) -> dict:
        return read_tallies(self.grid, self.tally.data_ptr(), self.J, self.nfaces, self.stream())

    def run(self, n_packets: int, seed: int, **kw) -> dict:
        self.reset()
        self.launch(n_packets, seed, **kw)
        return self.read()

    def redistribution(self, n_sub: int = 3):
        """Device thresholds of eq. R_discrete for this grid (uint32 tensor, J x (J-1)),
        for launch(..., redist=...) on a hybrid table."""
        torch = self.torch
        nb = redistribution_bytes(self.grid)
        buf = torch.empty(nb // 4, dtype=torch.int32, device=self.device)
        precompute_redistribution(self.grid, self.table.data_ptr(), n_sub, buf.data_ptr(), nb, self.stream())
        return buf

    def time_run(self, n_packets: int, seed: int, t_edges, max_steps: int = 0, chunk: int = 0,
                 threads_per_cta: int = 0, ctas_per_sm: int = 0, leaks: bool = False, regroup: int = 0) -> dict:
        """A flash of n_packets at the source at t_edges[0], advanced through the
        steps [t_edges[n], t_edges[n+1]], one launch per step.  Returns per step
        n: bins[n, s] (packets in state s = cell * J + bin at t_edges[n+1]),
        path[n, s] (path length spent in s during the step, ticks converted to
        length), esc[n], dwells[n], transitions[n], alive[n]; the walk's
        tallies; with leaks=True also leak[n, cell, face, io], the optical
        depths k dl of the leaks out of (io = 0) and into (io = 1) each face
        (eq. a_estimator)."""
        torch = self.torch
        te = np.asarray(t_edges, dtype=np.float64)
        nt = len(te) - 1
        S = int(self.w.ncell) * self.J
        need = time_state_bytes(n_packets)
        if need == 0:
            raise ValueError("n_packets out of range")
        state = torch.empty(need, dtype=torch.uint8, device=self.device)
        bins = torch.zeros((nt, S), dtype=torch.int64, device=self.device)
        path = torch.zeros((nt, S), dtype=torch.int64, device=self.device)
        counts = torch.zeros((nt, 5), dtype=torch.int64, device=self.device)
        nf = 2 * self.w.ndim
        leak = torch.zeros((nt, int(self.w.ncell) * nf * 2), dtype=torch.float64, device=self.device) if leaks \
            else None
        weighted = self.params.dust_abs > 0.0 and self.params.dust_method == DUST_WEIGHTS
        wb = torch.zeros((nt, S), dtype=torch.float64, device=self.device) if weighted else None
        wp = torch.zeros((nt, S), dtype=torch.float64, device=self.device) if weighted else None
        self.reset()
        for n in range(nt):
            st = TimeStep(seed, n_packets, max_steps, float(te[n]), float(te[n + 1]), 1 if n == 0 else 0, chunk,
                          threads_per_cta, ctas_per_sm, regroup)
            time_step_launch(self.grid, self.table.data_ptr(), st, state.data_ptr(), state.numel(),
                             self.tally.data_ptr(), self.tally.numel() * 8, bins[n].data_ptr(), path[n].data_ptr(),
                             counts[n].data_ptr(), self.stream(), leak[n].data_ptr() if leaks else 0,
                             wb[n].data_ptr() if weighted else 0, wp[n].data_ptr() if weighted else 0)
        c = counts.cpu().numpy().astype(np.uint64)
        ticks = path.cpu().numpy().astype(np.float64)
        out = dict(bins=bins.cpu().numpy().astype(np.uint64), path=ticks * (np.diff(te) / TIME_TICKS)[:, None],
                   path_ticks=path.cpu().numpy().astype(np.uint64), esc=c[:, 0], dwells=c[:, 1],
                   transitions=c[:, 2], alive=c[:, 3], absorbed=c[:, 4], tallies=self.read())
        if weighted:  # dust by weights: weighted bin and path (length) estimates
            out["wbins"] = wb.cpu().numpy()
            out["wpath"] = wp.cpu().numpy() * (np.diff(te) / TIME_TICKS)[:, None]
        if leaks:
            lk = leak.cpu().numpy() * (np.diff(te) / TIME_TICKS)[:, None]
            out["leak"] = lk.reshape(nt, int(self.w.ncell), nf, 2)
        return out

    def scatter(self, x_in: float, seed: int, n: int):
        out = self.torch.empty(n, dtype=self.torch.float32, device=self.device)
        scatter_samples(self.grid, self.table.data_ptr(), x_in, seed, n, out.data_ptr(), self.stream())
        return out.cpu().numpy().astype(np.float64)

    def packet_states(self, n_packets: int, first: int, count: int) -> dict:
        return read_packet_states(self.grid, self.state.data_ptr(), n_packets, first, count, self.stream())

    def rows(self):
        K = grid_sizes(self.grid, 1).n_outcomes  # one more with dust absorption
        return table_rows(self.grid, self.table.data_ptr(), self.w.ncell, self.J, K, self.stream())

    def close(self):
        destroy_grid(self.grid)
        self.grid = None

    def __del__(self):
        try:
            if self.grid:
                destroy_grid(self.grid)
        except Exception:
            pass


class Batch:
    """Many precomputed Problems walked by one persistent launch (C-ABI
    rddmc_batch_*): descriptors, tallies and scratch in torch device buffers."""

    def __init__(self, problems, n_packets, trial_fraction=0.01):
        import torch
        self.torch = torch
        self.problems = list(problems)
        self.device = self.problems[0].device
        n = len(self.problems)
        grids = (ctypes.c_void_p * n)(*[p.grid for p in self.problems])
        tables = (ctypes.c_void_p * n)(*[p.table.data_ptr() for p in self.problems])
        npk = (ctypes.c_uint64 * n)(*[int(v) for v in n_packets])
        h = ctypes.c_void_p()
        _check("rddmc_batch_create", lib().rddmc_batch_create(grids, tables, npk, n, ctypes.byref(h)))
        self.h = h.value
        db, tb, sb, tot = (ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64())
        _check("rddmc_batch_sizes", lib().rddmc_batch_sizes(ctypes.c_void_p(self.h), ctypes.byref(db),
                                                            ctypes.byref(tb), ctypes.byref(sb), ctypes.byref(tot)))
        self.total = tot.value
        self.desc = torch.empty(db.value, dtype=torch.uint8, device=self.device)
        self.tally = torch.zeros(tb.value // 8, dtype=torch.int64, device=self.device)
        self.scratch = torch.zeros(sb.value // 8, dtype=torch.int64, device=self.device)
        _check("rddmc_batch_upload", lib().rddmc_batch_upload(ctypes.c_void_p(self.h), float(trial_fraction),
                                                              ctypes.c_void_p(self.desc.data_ptr()),
                                                              self.desc.numel(), ctypes.c_void_p(self.stream())))

    def stream(self) -> int:
        return self.torch.cuda.current_stream(self.device).cuda_stream

    def launch(self, opts: RunOpts, trial: bool = False, reset: bool = True):
        if reset:
            self.tally.zero_()
        _check("rddmc_batch_launch", lib().rddmc_batch_launch(
            ctypes.c_void_p(self.h), ctypes.c_void_p(self.desc.data_ptr()), ctypes.byref(opts), int(trial),
            ctypes.c_void_p(self.scratch.data_ptr()), self.scratch.numel() * 8, ctypes.c_void_p(self.tally.data_ptr()),
            self.tally.numel() * 8, ctypes.c_void_p(self.stream())))

    def read(self, inst: int) -> dict:
        p = self.problems[inst]
        t = Tallies()
        hist = np.zeros(p.J + 2, dtype=np.uint64)
        faces = np.zeros(p.nfaces, dtype=np.uint64)
        sb = np.zeros(NSB, dtype=np.uint64)
        _check("rddmc_batch_read_tallies", lib().rddmc_batch_read_tallies(
            ctypes.c_void_p(self.h), ctypes.c_void_p(self.tally.data_ptr()), int(inst), ctypes.byref(t),
            _np_ptr(hist), _np_ptr(faces), _np_ptr(sb), ctypes.c_void_p(self.stream())))
        d = {k: int(getattr(t, k)) for k, _ in Tallies._fields_}
        d.update(hist=hist, faces=faces, sb=sb)
        return d

    def graph(self, opts: RunOpts) -> int:
        ge = ctypes.c_void_p()
        _check("rddmc_batch_graph_create", lib().rddmc_batch_graph_create(
            ctypes.c_void_p(self.h), ctypes.c_void_p(self.desc.data_ptr()), ctypes.byref(opts),
            ctypes.c_void_p(self.scratch.data_ptr()), self.scratch.numel() * 8,
            ctypes.c_void_p(self.tally.data_ptr()), self.tally.numel() * 8, ctypes.c_void_p(self.stream()),
            ctypes.byref(ge)))
        return ge.value

    def graph_launch(self, ge: int):
        _check("rddmc_batch_graph_launch", lib().rddmc_batch_graph_launch(ctypes.c_void_p(ge),
                                                                          ctypes.c_void_p(self.stream())))

    @staticmethod
    def graph_destroy(ge: int):
        lib().rddmc_batch_graph_destroy(ctypes.c_void_p(ge))

    def autotune(self, base: RunOpts):
        best = RunOpts()
        rate = ctypes.c_double()
        _check("rddmc_batch_autotune", lib().rddmc_batch_autotune(
            ctypes.c_void_p(self.h), ctypes.c_void_p(self.desc.data_ptr()), ctypes.byref(base),
            ctypes.c_void_p(self.scratch.data_ptr()), self.scratch.numel() * 8,
            ctypes.c_void_p(self.tally.data_ptr()), self.tally.numel() * 8, ctypes.c_void_p(self.stream()),
            ctypes.byref(best), ctypes.byref(rate)))
        return best, rate.value

    def __del__(self):
        try:
            if self.h:
                lib().rddmc_batch_destroy(ctypes.c_void_p(self.h))
        except Exception:
            pass


# ----------------------------------------------------------------------------- learned exit proposal
def cell_tau(grid, d_table: int, cell: int, J: int, stream: int = 0) -> np.ndarray:
    out = np.zeros(J, dtype=np.float32)
    _check("rddmc_cell_tau", lib().rddmc_cell_tau(ctypes.c_void_p(grid), ctypes.c_void_p(d_table), int(cell),
                                                  _np_ptr(out), ctypes.c_void_p(stream)))
    return out


def fp_generate(grids, d_tables, b, jlo, jhi, seed, p0, n, cap, d_out, d_steps, train=None, stream=0):
    """First passages through a uniform brick: d_out receives 8 int32 per
    sample (rddmc_fp_generate)."""
    L = len(grids)
    g = (ctypes.c_void_p * L)(*grids)
    t = (ctypes.c_void_p * L)(*d_tables)
    lo = np.ascontiguousarray(jlo, dtype=np.int32)
    hi = np.ascontiguousarray(jhi, dtype=np.int32)
    _check("rddmc_fp_generate", lib().rddmc_fp_generate(
        g, t, int(L), int(b), _np_ptr(lo), _np_ptr(hi), int(seed), int(p0), int(n), int(cap), ctypes.c_void_p(d_out),
        ctypes.c_void_p(d_steps), ctypes.byref(train) if train is not None else None, ctypes.c_void_p(stream)))


def fp_region_generate(grid, d_table: int, region: FpRegion, seed: int, p0: int, n: int, cap: int, d_out: int,
                       d_steps: int, train: Optional[FpTrain] = None, stream: int = 0):
    """rddmc_fp_region_generate: first passages out of regions of the grid's own medium."""
    _check("rddmc_fp_region_generate", lib().rddmc_fp_region_generate(
        ctypes.c_void_p(grid), ctypes.c_void_p(d_table), ctypes.byref(region), int(seed), int(p0), int(n), int(cap),
        ctypes.c_void_p(d_out), ctypes.c_void_p(d_steps), ctypes.byref(train) if train is not None else None,
        ctypes.c_void_p(stream)))


def mlp_param_count(n_out: int) -> int:
    return int(lib().rddmc_mlp_param_count(int(n_out)))


def mlp_work_bytes(batch: int, n_out: int) -> int:
    return int(lib().rddmc_mlp_work_bytes(int(batch), int(n_out)))


def mlp_to_bf16(n_out, d_wf, d_wb, stream=0):
    _check("rddmc_mlp_to_bf16", lib().rddmc_mlp_to_bf16(int(n_out), ctypes.c_void_p(d_wf), ctypes.c_void_p(d_wb),
                                                        ctypes.c_void_p(stream)))


def mlp_forward(n_out, d_wf, d_wb, d_x, batch, d_work, d_logits, stream=0):
    _check("rddmc_mlp_forward", lib().rddmc_mlp_forward(int(n_out), ctypes.c_void_p(d_wf), ctypes.c_void_p(d_wb),
                                                        ctypes.c_void_p(d_x), int(batch), ctypes.c_void_p(d_work),
                                                        ctypes.c_void_p(d_logits), ctypes.c_void_p(stream)))


def mlp_loss_grad(n_out, nA, nB, d_wf, d_wb, d_x, d_ta, d_tb, batch, d_work, d_grad, d_loss, stream=0, nC=0, S=0,
                  d_tc=0):
    _check("rddmc_mlp_loss_grad", lib().rddmc_mlp_loss_grad(
        int(n_out), int(nA), int(nB), int(nC), int(S), ctypes.c_void_p(d_wf), ctypes.c_void_p(d_wb),
        ctypes.c_void_p(d_x), ctypes.c_void_p(d_ta), ctypes.c_void_p(d_tb), ctypes.c_void_p(d_tc or None), int(batch),
        ctypes.c_void_p(d_work), ctypes.c_void_p(d_grad), ctypes.c_void_p(d_loss), ctypes.c_void_p(stream)))


def mlp_status(stream=0):
    """Synchronise and raise if a tensor-core product's bounded wait ran out."""
    _check("rddmc_mlp_status", lib().rddmc_mlp_status(ctypes.c_void_p(stream)))


def mlp_adam(n_out, d_wf, d_wb, d_grad, d_m, d_v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=0):
    _check("rddmc_mlp_adam", lib().rddmc_mlp_adam(
        int(n_out), ctypes.c_void_p(d_wf), ctypes.c_void_p(d_wb), ctypes.c_void_p(d_grad), ctypes.c_void_p(d_m),
        ctypes.c_void_p(d_v), int(step), float(lr), float(beta1), float(beta2), float(eps), ctypes.c_void_p(stream)))


def propose(grid, d_table, proposal: Proposal, seed, n_packets, d_state, d_tallies, n_out, nA, nB, d_wf, d_wb, batch,
            d_work, stream=0, nC=0) -> int:
    served = ctypes.c_uint64()
    _check("rddmc_propose", lib().rddmc_propose(
        ctypes.c_void_p(grid), ctypes.c_void_p(d_table), ctypes.byref(proposal), int(seed), int(n_packets),
        ctypes.c_void_p(d_state), ctypes.c_void_p(d_tallies), int(n_out), int(nA), int(nB), int(nC),
        ctypes.c_void_p(d_wf),
        ctypes.c_void_p(d_wb), int(batch), ctypes.c_void_p(d_work), ctypes.byref(served), ctypes.c_void_p(stream)))
    return served.value
