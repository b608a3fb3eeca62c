"""Python binding of libepsr (ctypes): argument marshalling only.

Every function here has the name of the C entry point it calls (include/epsr.h) and
takes torch tensors for device buffers (passed as raw pointers) and NumPy arrays or
Python numbers for host data. All computation happens in the CUDA library; there is no
CPU fallback: if libepsr.so is missing or CUDA is unavailable, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libepsr.so")
PROBE_LIB_PATH = os.path.join(_HERE, "libepsr_probe.so")
# Every symbol include/epsr_probe.h declares (the measurement library of the benchmark).
PROBE_EXPORTS = ["epsr_bench_barrier_floor", "epsr_bench_alu_rate"]

EPSR_OK, EPSR_EINVAL, EPSR_ENOMEM, EPSR_ECUDA, EPSR_ELAUNCH, EPSR_ETIMEOUT, EPSR_ENUMERIC = range(7)
MAX_TYPES = 8
MAX_MOL_ATOMS = 8
MOVE_ATOM, MOVE_RIGID_MOLECULE, MOVE_FLEXIBLE_MOLECULE = 0, 1, 2
SQ_FP32, SQ_TF32X3, SQ_BF16X3, SQ_BF16X6 = 0, 1, 2, 3

# Every symbol include/epsr.h declares (checked by the CPU test suite).
EXPORTS = [
    "epsr_strerror", "epsr_last_error_detail", "epsr_version",
    "epsr_box_create", "epsr_batch_create", "epsr_box_destroy", "epsr_box_info",
    "epsr_box_offsets", "epsr_box_get_coords", "epsr_box_set_coords",
    "epsr_box_set_coords_device", "epsr_box_get_coords_device", "epsr_box_set_ep",
    "epsr_box_get_ep", "epsr_box_total_energy", "epsr_mc_sweep", "epsr_mc_stats_get",
    "epsr_mc_sweep_async", "epsr_mc_status",
    "epsr_mc_set_batch", "epsr_mc_set_ctas", "epsr_debug_barrier_fault",
    "epsr_partial_gr", "epsr_partial_gr_tiles", "epsr_partial_gr_range", "epsr_normalize_g",
    "epsr_sq_weights", "epsr_sq_plan_create", "epsr_sq_plan_destroy", "epsr_sq_exec", "epsr_sq",
    "epsr_noalloc_scratch_bytes", "epsr_partial_gr_noalloc", "epsr_ep_update",
    "epsr_gr_smeared_fwd", "epsr_gr_smeared_bwd", "epsr_sq_exec_adjoint", "epsr_chi2",
    "epsr_checkpoint_size", "epsr_checkpoint_save", "epsr_checkpoint_load", "epsr_launch_count",
    "epsr_mc_set_cells", "epsr_sq_plan_status", "epsr_partial_gr_cells",
    "epsr_sq_plan_set_tiles",
    "epsr_sq_plan_get_tiles", "epsr_gr_set_ctas_per_sm", "epsr_box_get_launch", "epsr_autotune",
    "epsr_sq_plan_autotune", "epsr_refiner_create", "epsr_refine_step", "epsr_refiner_get",
    "epsr_refiner_destroy",
]


class BoxDesc(C.Structure):
    _fields_ = [("n_atoms", C.c_int64), ("n_mol", C.c_int64), ("L_fx", C.c_int64),
                ("scale_log2", C.c_int32), ("n_types", C.c_int32),
                ("q", C.c_double * MAX_TYPES), ("sigma", C.c_double * MAX_TYPES),
                ("eps", C.c_double * MAX_TYPES), ("b", C.c_double * MAX_TYPES),
                ("r_coul", C.c_double), ("bin_p", C.c_int32), ("bin_q", C.c_int32),
                ("n_bins", C.c_int32), ("move_kind", C.c_int32), ("temperature", C.c_double),
                ("max_translation", C.c_double), ("max_rotation_deg", C.c_double),
                ("bond_k", C.c_double * (MAX_TYPES * MAX_TYPES)),
                ("bond_d", C.c_double * (MAX_TYPES * MAX_TYPES)), ("r_lj", C.c_double)]


class Tuning(C.Structure):
    _fields_ = [("mc_batch", C.c_int32), ("mc_ctas", C.c_int32), ("gr_ctas_per_sm", C.c_int32),
                ("from_cache", C.c_int32), ("mc_us_per_move", C.c_double), ("gr_ms", C.c_double)]


class RefineParams(C.Structure):
    _fields_ = [("moves_per_pass", C.c_int64), ("seed", C.c_uint64), ("move0", C.c_uint64),
                ("accumulate", C.c_int32), ("n_basis", C.c_int32), ("s_basis", C.c_double),
                ("gamma", C.c_double), ("alpha", C.c_double)]


class RefineResult(C.Structure):
    _fields_ = [("iteration", C.c_int64), ("attempted", C.c_int64), ("accepted", C.c_int64),
                ("n_configs", C.c_int64), ("next_move", C.c_uint64), ("chi2", C.c_double),
                ("ep_change_max", C.c_double)]


class McStats(C.Structure):
    _fields_ = [("attempted", C.c_int64), ("accepted", C.c_int64), ("nonfinite", C.c_int64),
                ("sum_dU", C.c_double)]


MOVE_LOG_DTYPE = np.dtype([("mol", np.int32), ("accepted", np.int32), ("dU", np.float32),
                           ("n_atoms", np.int32), ("u_acc", np.float64),
                           ("trial", np.int32, (MAX_MOL_ATOMS, 3)), ("pad", np.int32, (2,))])
assert MOVE_LOG_DTYPE.itemsize == 128


class EpsrError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: {detail or 'error'} (status {status})")
        self.status = status


_lib = None


def lib():
    """Load libepsr.so (built in-tree by __graft_entry__.build or build.py)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libepsr.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, u64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
        P = C.POINTER
        sig = {
            "epsr_strerror": ([C.c_int], C.c_char_p),
            "epsr_last_error_detail": ([C.c_char_p, C.c_size_t], C.c_int),
            "epsr_version": ([], C.c_int),
            "epsr_box_create": ([P(BoxDesc), vp, vp, vp, vp, P(vp)], C.c_int),
            "epsr_batch_create": ([P(BoxDesc), i32, vp, vp, vp, vp, P(vp)], C.c_int),
            "epsr_box_destroy": ([vp], C.c_int),
            "epsr_box_info": ([vp, P(i32), P(i64), P(i64)], C.c_int),
            "epsr_box_offsets": ([vp, i32, P(i64), P(i64)], C.c_int),
            "epsr_box_get_coords": ([vp, vp, vp], C.c_int),
            "epsr_box_set_coords": ([vp, vp, vp], C.c_int),
            "epsr_box_set_coords_device": ([vp, vp, vp], C.c_int),
            "epsr_box_get_coords_device": ([vp, vp, vp], C.c_int),
            "epsr_box_set_ep": ([vp, i32, vp, vp], C.c_int),
            "epsr_box_get_ep": ([vp, i32, vp, vp], C.c_int),
            "epsr_box_total_energy": ([vp, vp, vp], C.c_int),
            "epsr_mc_sweep": ([vp, i64, u64, u64, vp, vp, vp], C.c_int),
            "epsr_mc_stats_get": ([vp, vp, vp], C.c_int),
            "epsr_mc_sweep_async": ([vp, i64, u64, u64, vp, vp], C.c_int),
            "epsr_mc_status": ([vp, P(i32), vp], C.c_int),
            "epsr_mc_set_batch": ([vp, i32], C.c_int),
            "epsr_mc_set_ctas": ([vp, i32], C.c_int),
            "epsr_debug_barrier_fault": ([vp, i32, dbl], C.c_int),
            "epsr_partial_gr": ([vp, vp, vp, i64, vp], C.c_int),
            "epsr_partial_gr_cells": ([vp, vp, vp, i64, vp], C.c_int),
            "epsr_partial_gr_tiles": ([vp, P(i64)], C.c_int),
            "epsr_partial_gr_range": ([vp, i64, i64, vp, vp], C.c_int),
            "epsr_normalize_g": ([vp, vp, vp, i64, vp], C.c_int),
            "epsr_sq_weights": ([vp, i32, vp, vp], C.c_int),
            "epsr_sq_plan_create": ([vp, i32, i32, dbl, i32, i32, vp, P(vp)], C.c_int),
            "epsr_sq_plan_destroy": ([vp], C.c_int),
            "epsr_sq_exec": ([vp, vp, i32, vp, i32, vp, vp, vp, vp], C.c_int),
            "epsr_sq": ([vp, i32, i32, dbl, vp, i32, vp, i32, vp, vp, vp, i32, vp], C.c_int),
            "epsr_noalloc_scratch_bytes": ([], C.c_size_t),
            "epsr_ep_update": ([vp, i32, vp, i32, vp, vp, i32, i32, dbl, dbl, dbl, vp, vp], C.c_int),
            "epsr_gr_smeared_fwd": ([vp, dbl, vp, vp, vp], C.c_int),
            "epsr_checkpoint_size": ([vp, P(C.c_size_t)], C.c_int),
            "epsr_launch_count": ([P(C.c_uint64)], C.c_int),
            "epsr_mc_set_cells": ([vp, C.c_int32, C.c_int32], C.c_int),
            "epsr_sq_plan_status": ([vp, P(C.c_int32), vp], C.c_int),
            "epsr_checkpoint_save": ([vp, vp, C.c_size_t, vp], C.c_int),
            "epsr_checkpoint_load": ([vp, vp, C.c_size_t, vp], C.c_int),
            "epsr_gr_smeared_bwd": ([vp, dbl, vp, vp, vp], C.c_int),
            "epsr_sq_exec_adjoint": ([vp, vp, i32, vp, i32, vp, vp], C.c_int),
            "epsr_chi2": ([vp, vp, vp, vp, i32, vp, i32, dbl, dbl, vp, vp, vp, vp], C.c_int),
            "epsr_partial_gr_noalloc": ([vp, vp, i64, i64, i32, i32, i32, i32, i32, vp, vp], C.c_int),
            "epsr_sq_plan_set_tiles": ([vp, i32, i32], C.c_int),
            "epsr_gr_set_ctas_per_sm": ([vp, i32], C.c_int),
            "epsr_refiner_create": ([vp, vp, vp, i32, vp, vp, vp, i32, P(RefineParams), vp, P(vp)], C.c_int),
            "epsr_refine_step": ([vp, vp, P(RefineResult), vp], C.c_int),
            "epsr_refiner_get": ([vp, vp, vp, vp, vp, vp, vp], C.c_int),
            "epsr_refiner_destroy": ([vp], C.c_int),
            "epsr_box_get_launch": ([vp, P(C.c_int32), P(C.c_int32), P(C.c_int32)], C.c_int),
            "epsr_autotune": ([vp, C.c_uint64, i32, P(Tuning), vp], C.c_int),
            "epsr_sq_plan_autotune": ([vp, vp, i32, vp, i32, vp, vp, vp, P(C.c_int32), P(C.c_int32),
                                       P(C.c_double), vp], C.c_int),
            "epsr_sq_plan_get_tiles": ([vp, i32, i32, i32, P(C.c_int32), P(C.c_int32)], C.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(status: int, where: str):
    if status != EPSR_OK:
        buf = C.create_string_buffer(512)
        lib().epsr_last_error_detail(buf, 512)
        raise EpsrError(status, where, buf.value.decode(errors="replace"))


def _np_ptr(a: np.ndarray):
    return C.c_void_p(a.ctypes.data)


def _dev_ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _buf(t, dtypes, min_numel: int, name: str):
    """Device pointer of a caller buffer that a kernel writes: checks its element type, its
    length and that it lives on the current device, so that a short or misplaced buffer is a
    ValueError here instead of an out-of-bounds write on the GPU."""
    if t is None:
        return None
    import torch
    if t.dtype not in dtypes:
        raise ValueError(f"{name}: expected dtype {' or '.join(str(d) for d in dtypes)}, got {t.dtype}")
    if t.numel() < min_numel:
        raise ValueError(f"{name}: {t.numel()} elements, at least {min_numel} needed")
    if t.is_cuda and t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name}: on cuda:{t.device.index}, the current device is "
                         f"cuda:{torch.cuda.current_device()}")
    return _dev_ptr(t)


def _hist_ptr(t, n: int, name: str = "hist"):
    import torch
    return _buf(t, (torch.int64, torch.uint64), n, name)


def _g_ptr(t, n: int, name: str = "g"):
    import torch
    return _buf(t, (torch.float32,), n, name)


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def box_desc(system) -> BoxDesc:
    """epsr_box_desc of a synth.System (plain field copy)."""
    d = BoxDesc()
    d.n_atoms = system.n_atoms
    d.n_mol = system.n_mol
    d.L_fx = system.L_fx
    d.scale_log2 = 20
    d.n_types = system.n_types
    for i in range(system.n_types):
        d.q[i], d.sigma[i], d.eps[i], d.b[i] = (system.q[i], system.sigma[i], system.eps[i],
                                                system.b[i])
    d.r_coul = system.r_coul
    d.bin_p, d.bin_q, d.n_bins = system.bin_p, system.bin_q, system.n_bins
    d.move_kind = MOVE_RIGID_MOLECULE if system.rigid_molecules else MOVE_ATOM
    if getattr(system, "flexible", False):
        d.move_kind = MOVE_FLEXIBLE_MOLECULE
        for a in range(system.n_types):
            for b in range(system.n_types):
                d.bond_k[a * MAX_TYPES + b] = float(system.bond_k[a][b])
                d.bond_d[a * MAX_TYPES + b] = float(system.bond_d[a][b])
    d.temperature = system.temperature
    d.max_translation = system.max_translation
    d.max_rotation_deg = system.max_rotation_deg
    d.r_lj = float(getattr(system, "r_lj", 0.0))
    return d


def epsr_strerror(status: int) -> str:
    return lib().epsr_strerror(status).decode()


def epsr_version() -> int:
    return lib().epsr_version()


_probe = None


def probe_lib():
    """libepsr_probe.so: the GPU measurements of the benchmark (grid-barrier floor, issue rates),
    kept out of the product library; it links against libepsr.so, loaded first."""
    global _probe
    if _probe is None:
        lib()
        if not os.path.exists(PROBE_LIB_PATH):
            raise RuntimeError(f"libepsr_probe.so not built ({PROBE_LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(PROBE_LIB_PATH)
        L.epsr_bench_barrier_floor.argtypes = [C.c_int32, C.c_int32, C.POINTER(C.c_double), C.c_void_p]
        L.epsr_bench_barrier_floor.restype = C.c_int
        L.epsr_bench_alu_rate.argtypes = [C.c_int32, C.POINTER(C.c_double), C.c_void_p]
        L.epsr_bench_alu_rate.restype = C.c_int
        _probe = L
    return _probe


def epsr_bench_barrier_floor(ctas: int, iters: int = 2000, stream=None) -> float:
    """ns per grid barrier of the sweep's exchange with `ctas` co-resident CTAs."""
    v = C.c_double()
    _check(probe_lib().epsr_bench_barrier_floor(ctas, iters, C.byref(v), _stream(stream)), "epsr_bench_barrier_floor")
    return v.value


def epsr_bench_alu_rate(kind: int, stream=None) -> float:
    """Lane-operations/s: kind 0 = int32 adds, 1 = FP32 FMAs."""
    v = C.c_double()
    _check(probe_lib().epsr_bench_alu_rate(kind, C.byref(v), _stream(stream)), "epsr_bench_alu_rate")
    return v.value


def epsr_launch_count() -> int:
    n = C.c_uint64()
    _check(lib().epsr_launch_count(C.byref(n)), "epsr_launch_count")
    return n.value


class Box:
    """Owner of an epsr_box handle (one box or a batch of replicas)."""

    def __init__(self, systems, stream=None):
        systems = systems if isinstance(systems, (list, tuple)) else [systems]
        self.systems = list(systems)
        descs = (BoxDesc * len(systems))(*[box_desc(s) for s in systems])
        xyz = np.ascontiguousarray(np.concatenate([s.xyz for s in systems]), np.int32)
        typ = np.ascontiguousarray(np.concatenate([s.type for s in systems]), np.int32)
        ms = np.ascontiguousarray(np.concatenate([s.mol_start for s in systems]), np.int64)
        h = C.c_void_p()
        if len(systems) == 1:
            st = lib().epsr_box_create(descs, _np_ptr(xyz), _np_ptr(typ), _np_ptr(ms),
                                       _stream(stream), C.byref(h))
            _check(st, "epsr_box_create")
        else:
            st = lib().epsr_batch_create(descs, len(systems), _np_ptr(xyz), _np_ptr(typ),
                                         _np_ptr(ms), _stream(stream), C.byref(h))
            _check(st, "epsr_batch_create")
        self.h = h
        nb, na, hl = C.c_int32(), C.c_int64(), C.c_int64()
        _check(lib().epsr_box_info(h, C.byref(nb), C.byref(na), C.byref(hl)), "epsr_box_info")
        self.n_boxes, self.n_atoms, self.hist_len = nb.value, na.value, hl.value

    def close(self):
        if getattr(self, "h", None):
            lib().epsr_box_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- layout ------------------------------------------------------------------------
    def epsr_box_offsets(self, b: int):
        ho, ao = C.c_int64(), C.c_int64()
        _check(lib().epsr_box_offsets(self.h, b, C.byref(ho), C.byref(ao)), "epsr_box_offsets")
        return ho.value, ao.value

    # -- coordinates and tables ------------------------------------------------------------
    def epsr_box_get_coords(self, stream=None) -> np.ndarray:
        out = np.zeros((self.n_atoms, 3), np.int32)
        _check(lib().epsr_box_get_coords(self.h, _np_ptr(out), _stream(stream)), "epsr_box_get_coords")
        return out

    def epsr_box_set_coords(self, xyz: np.ndarray, stream=None):
        x = np.ascontiguousarray(xyz, np.int32)
        _check(lib().epsr_box_set_coords(self.h, _np_ptr(x), _stream(stream)), "epsr_box_set_coords")

    def epsr_box_set_coords_device(self, xyz_dev, stream=None):
        _check(lib().epsr_box_set_coords_device(self.h, _dev_ptr(xyz_dev), _stream(stream)),
               "epsr_box_set_coords_device")

    def epsr_box_get_coords_device(self, xyz_dev, stream=None):
        _check(lib().epsr_box_get_coords_device(self.h, _dev_ptr(xyz_dev), _stream(stream)),
               "epsr_box_get_coords_device")

    def epsr_box_set_ep(self, b: int, ep: np.ndarray, stream=None):
        e = np.ascontiguousarray(ep, np.float32)
        _check(lib().epsr_box_set_ep(self.h, b, _np_ptr(e), _stream(stream)), "epsr_box_set_ep")

    def epsr_box_get_ep(self, b: int, shape, stream=None) -> np.ndarray:
        e = np.zeros(shape, np.float32)
        _check(lib().epsr_box_get_ep(self.h, b, _np_ptr(e), _stream(stream)), "epsr_box_get_ep")
        return e

    def epsr_box_total_energy(self, stream=None) -> np.ndarray:
        U = np.zeros(self.n_boxes, np.float64)
        _check(lib().epsr_box_total_energy(self.h, _np_ptr(U), _stream(stream)),
               "epsr_box_total_energy")
        return U

    # -- Monte Carlo ----------------------------------------------------------------------------
    def epsr_mc_sweep(self, n_moves: int, seed: int, move0: int = 0, log=None, stream=None):
        stats = (McStats * self.n_boxes)()
        _check(lib().epsr_mc_sweep(self.h, n_moves, seed, move0, stats, _dev_ptr(log),
                                   _stream(stream)), "epsr_mc_sweep")
        return [(s.attempted, s.accepted, s.nonfinite, s.sum_dU) for s in stats]

    def epsr_mc_sweep_async(self, n_moves: int, seed: int, move0: int = 0, log=None, stream=None):
        _check(lib().epsr_mc_sweep_async(self.h, n_moves, seed, move0, _dev_ptr(log),
                                         _stream(stream)), "epsr_mc_sweep_async")

    def epsr_mc_status(self, stream=None) -> int:
        st = C.c_int32()
        _check(lib().epsr_mc_status(self.h, C.byref(st), _stream(stream)), "epsr_mc_status")
        return st.value

    def epsr_mc_stats_get(self, stream=None):
        stats = (McStats * self.n_boxes)()
        _check(lib().epsr_mc_stats_get(self.h, stats, _stream(stream)), "epsr_mc_stats_get")
        return [(s.attempted, s.accepted, s.nonfinite, s.sum_dU) for s in stats]

    def epsr_mc_set_batch(self, k: int):
        _check(lib().epsr_mc_set_batch(self.h, k), "epsr_mc_set_batch")

    def epsr_mc_set_cells(self, margin_fx: int, escapee_cap: int = -1):
        _check(lib().epsr_mc_set_cells(self.h, margin_fx, escapee_cap), "epsr_mc_set_cells")

    def epsr_mc_set_ctas(self, n: int):
        _check(lib().epsr_mc_set_ctas(self.h, n), "epsr_mc_set_ctas")

    def epsr_gr_set_ctas_per_sm(self, n: int):
        _check(lib().epsr_gr_set_ctas_per_sm(self.h, n), "epsr_gr_set_ctas_per_sm")

    def epsr_box_get_launch(self):
        b, c, g = C.c_int32(), C.c_int32(), C.c_int32()
        _check(lib().epsr_box_get_launch(self.h, C.byref(b), C.byref(c), C.byref(g)), "epsr_box_get_launch")
        return {"mc_batch": b.value, "mc_ctas": c.value, "gr_ctas_per_sm": g.value}

    def epsr_autotune(self, seed: int = 12345, probe_moves: int = 0, stream=None) -> dict:
        """Times the sweep and histogram launch shapes on this handle and applies the fastest
        (state saved and restored around the probes); returns the chosen settings."""
        t = Tuning()
        _check(lib().epsr_autotune(self.h, seed, probe_moves, C.byref(t), _stream(stream)), "epsr_autotune")
        return {f: getattr(t, f) for f, _ in Tuning._fields_}

    def epsr_debug_barrier_fault(self, cta: int, timeout_ms: float):
        _check(lib().epsr_debug_barrier_fault(self.h, cta, timeout_ms), "epsr_debug_barrier_fault")

    # -- histograms -------------------------------------------------------------------------------
    def epsr_partial_gr(self, hist, g=None, n_configs: int = 1, stream=None):
        _check(lib().epsr_partial_gr(self.h, _hist_ptr(hist, self.hist_len),
                                     _g_ptr(g, self.hist_len), n_configs, _stream(stream)),
               "epsr_partial_gr")

    def epsr_partial_gr_cells(self, hist, g=None, n_configs: int = 1, stream=None):
        _check(lib().epsr_partial_gr_cells(self.h, _hist_ptr(hist, self.hist_len),
                                           _g_ptr(g, self.hist_len), n_configs, _stream(stream)),
               "epsr_partial_gr_cells")

    def epsr_partial_gr_tiles(self) -> int:
        n = C.c_int64()
        _check(lib().epsr_partial_gr_tiles(self.h, C.byref(n)), "epsr_partial_gr_tiles")
        return n.value

    def epsr_partial_gr_range(self, t0: int, t1: int, hist, stream=None):
        _check(lib().epsr_partial_gr_range(self.h, t0, t1, _hist_ptr(hist, self.hist_len),
                                           _stream(stream)), "epsr_partial_gr_range")

    def epsr_normalize_g(self, hist, g, n_configs: int = 1, stream=None):
        _check(lib().epsr_normalize_g(self.h, _hist_ptr(hist, self.hist_len),
                                      _g_ptr(g, self.hist_len), n_configs, _stream(stream)),
               "epsr_normalize_g")

    def epsr_ep_update(self, b: int, dS, w: np.ndarray, Q: np.ndarray, n_basis: int = 20,
                       s_basis: float = 0.5, gamma: float = 0.0, alpha: float = 1.0, stream=None):
        """Fit the Poisson basis to the pair-resolved Delta S and add it to box b's table;
        returns the coefficients C [P][n_basis]."""
        w = np.ascontiguousarray(w, np.float64)
        q = np.ascontiguousarray(Q, np.float32)
        P = self.systems[b].n_types * (self.systems[b].n_types + 1) // 2
        C_ = np.zeros((P, n_basis), np.float64)
        _check(lib().epsr_ep_update(self.h, b, _dev_ptr(dS), dS.shape[0], _np_ptr(w), _np_ptr(q),
                                    len(q), n_basis, s_basis, gamma, alpha, _np_ptr(C_),
                                    _stream(stream)), "epsr_ep_update")
        return C_

    def epsr_checkpoint_save(self, stream=None) -> bytes:
        n = C.c_size_t()
        _check(lib().epsr_checkpoint_size(self.h, C.byref(n)), "epsr_checkpoint_size")
        buf = (C.c_char * n.value)()
        _check(lib().epsr_checkpoint_save(self.h, buf, n.value, _stream(stream)), "epsr_checkpoint_save")
        return bytes(buf)

    def epsr_checkpoint_load(self, data: bytes, stream=None):
        buf = (C.c_char * len(data)).from_buffer_copy(data)
        _check(lib().epsr_checkpoint_load(self.h, buf, len(data), _stream(stream)), "epsr_checkpoint_load")

    def epsr_gr_smeared_fwd(self, sigma: float, Ht, gt=None, stream=None):
        _check(lib().epsr_gr_smeared_fwd(self.h, sigma, _dev_ptr(Ht), _dev_ptr(gt), _stream(stream)),
               "epsr_gr_smeared_fwd")

    def epsr_gr_smeared_bwd(self, sigma: float, dgt, grad, stream=None):
        _check(lib().epsr_gr_smeared_bwd(self.h, sigma, _dev_ptr(dgt), _dev_ptr(grad), _stream(stream)),
               "epsr_gr_smeared_bwd")

    def epsr_sq_weights(self, b: int):
        P = self.systems[b].n_types * (self.systems[b].n_types + 1) // 2
        w = np.zeros(P, np.float64)
        flat = np.zeros(1, np.float64)
        _check(lib().epsr_sq_weights(self.h, b, _np_ptr(w), _np_ptr(flat)), "epsr_sq_weights")
        return w, float(flat[0])


class SqPlan:
    """Owner of an epsr_sq_plan (cached sine-transform matrix for one Q grid)."""

    def __init__(self, Q: np.ndarray, n_bins: int, dr: float, mode: int = SQ_FP32,
                 max_cols: int = 64, stream=None):
        q = np.ascontiguousarray(Q, np.float32)
        h = C.c_void_p()
        _check(lib().epsr_sq_plan_create(_np_ptr(q), len(q), n_bins, dr, mode, max_cols,
                                         _stream(stream), C.byref(h)), "epsr_sq_plan_create")
        self.h, self.nQ, self.n_bins, self.mode = h, len(q), n_bins, mode

    def close(self):
        if getattr(self, "h", None):
            lib().epsr_sq_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def epsr_sq_plan_status(self, stream=None) -> int:
        st = C.c_int32()
        _check(lib().epsr_sq_plan_status(self.h, C.byref(st), _stream(stream)), "epsr_sq_plan_status")
        return st.value

    def epsr_sq_plan_set_tiles(self, n_chunk: int, k_split: int):
        _check(lib().epsr_sq_plan_set_tiles(self.h, n_chunk, k_split), "epsr_sq_plan_set_tiles")

    def epsr_sq_plan_autotune(self, g, w: np.ndarray, cols_per_set: int, flat: np.ndarray,
                              S_partial=None, S_total=None, stream=None) -> dict:
        """Times the tensor-core tilings of this exec and sets the fastest on the plan."""
        w = np.ascontiguousarray(w, np.float64)
        flat = np.ascontiguousarray(np.atleast_1d(flat), np.float64)
        nc, ks, us = C.c_int32(), C.c_int32(), C.c_double()
        _check(lib().epsr_sq_plan_autotune(self.h, _dev_ptr(g), g.shape[0], _np_ptr(w), cols_per_set,
                                           _np_ptr(flat), _dev_ptr(S_partial), _dev_ptr(S_total),
                                           C.byref(nc), C.byref(ks), C.byref(us), _stream(stream)),
               "epsr_sq_plan_autotune")
        return {"cols_per_cta": nc.value, "k_split": ks.value, "us": us.value}

    def epsr_sq_plan_get_tiles(self, n_cols: int, cols_per_set: int, with_totals: bool = True):
        nc, ks = C.c_int32(), C.c_int32()
        _check(lib().epsr_sq_plan_get_tiles(self.h, n_cols, cols_per_set, int(with_totals),
                                            C.byref(nc), C.byref(ks)), "epsr_sq_plan_get_tiles")
        return nc.value, ks.value

    def epsr_sq_exec(self, g, w: np.ndarray, cols_per_set: int, flat: np.ndarray,
                     S_partial=None, S_total=None, stream=None):
        w = np.ascontiguousarray(w, np.float64)
        flat = np.ascontiguousarray(np.atleast_1d(flat), np.float64)
        n_cols = g.shape[0]
        _check(lib().epsr_sq_exec(self.h, _dev_ptr(g), n_cols, _np_ptr(w), cols_per_set,
                                  _np_ptr(flat), _dev_ptr(S_partial), _dev_ptr(S_total),
                                  _stream(stream)), "epsr_sq_exec")


def _plan_adjoint(plan, dS_total, w, cols_per_set, dg, stream=None):
    w = np.ascontiguousarray(w, np.float64)
    _check(lib().epsr_sq_exec_adjoint(plan.h, _dev_ptr(dS_total), dg.shape[0], _np_ptr(w), cols_per_set,
                                      _dev_ptr(dg), _stream(stream)), "epsr_sq_exec_adjoint")


def _plan_chi2(plan, S, target, W, C, s_basis, rho, chi2, dS, dC, stream=None):
    W = np.ascontiguousarray(W, np.float64)
    n_basis = C.shape[1] if C is not None else 0
    _check(lib().epsr_chi2(plan.h, _dev_ptr(S), _dev_ptr(target), _np_ptr(W), len(W), _dev_ptr(C),
                           n_basis, s_basis, rho, _dev_ptr(chi2), _dev_ptr(dS), _dev_ptr(dC),
                           _stream(stream)), "epsr_chi2")


SqPlan.epsr_sq_exec_adjoint = _plan_adjoint
SqPlan.epsr_chi2 = _plan_chi2


def smeared_chi2_function():
    """torch.autograd.Function for chi^2(x, C) of the differentiable form: forward runs
    epsr_gr_smeared_fwd -> epsr_sq_exec -> epsr_chi2, backward runs epsr_sq_exec_adjoint ->
    epsr_gr_smeared_bwd. The positions are the box's own; `pos` is the tensor the gradient
    dchi2/dx (per Angstrom, [n_atoms][3]) is returned for. Only the upstream gradient is
    applied in torch (a scalar scale)."""
    import torch

    class SmearedChi2(torch.autograd.Function):
        @staticmethod
        def forward(ctx, pos, C_, box, plan, sigma, W, w_cols, flat, target, s_basis, rho):
            dev = pos.device
            P = len(W)
            Ht = torch.empty(box.hist_len, dtype=torch.float64, device=dev)
            gt = torch.empty(box.hist_len, dtype=torch.float32, device=dev)
            box.epsr_gr_smeared_fwd(sigma, Ht, gt)
            S = torch.empty((1, plan.nQ), dtype=torch.float32, device=dev)
            plan.epsr_sq_exec(gt.view(P, -1), w_cols, P, np.array([flat]), None, S)
            chi2 = torch.empty(1, dtype=torch.float64, device=dev)
            dS = torch.empty(plan.nQ, dtype=torch.float32, device=dev)
            dC = torch.empty_like(C_) if C_ is not None else None
            plan.epsr_chi2(S, target, W, C_.contiguous() if C_ is not None else None, s_basis, rho,
                           chi2, dS, dC)
            ctx.box, ctx.plan, ctx.sigma, ctx.w_cols, ctx.P = box, plan, sigma, w_cols, P
            ctx.save_for_backward(dS, dC if dC is not None else torch.empty(0, device=dev))
            ctx.has_C = C_ is not None
            ctx.S = S
            return chi2[0]

        @staticmethod
        def backward(ctx, gout):
            dS, dC = ctx.saved_tensors
            dev = dS.device
            dg = torch.empty((ctx.P, ctx.plan.n_bins), dtype=torch.float32, device=dev)
            ctx.plan.epsr_sq_exec_adjoint((dS * gout.float()).view(1, -1), ctx.w_cols, ctx.P, dg)
            grad = torch.empty((ctx.box.n_atoms, 3), dtype=torch.float32, device=dev)
            ctx.box.epsr_gr_smeared_bwd(ctx.sigma, dg, grad)
            gC = dC * gout if ctx.has_C else None
            return grad, gC, None, None, None, None, None, None, None, None, None

    return SmearedChi2


def epsr_sq(g, dr: float, Q: np.ndarray, w: np.ndarray, cols_per_set: int, flat: np.ndarray,
            S_partial=None, S_total=None, mode: int = SQ_FP32, stream=None):
    q = np.ascontiguousarray(Q, np.float32)
    w = np.ascontiguousarray(w, np.float64)
    flat = np.ascontiguousarray(np.atleast_1d(flat), np.float64)
    _check(lib().epsr_sq(_dev_ptr(g), g.shape[0], g.shape[1], dr, _np_ptr(q), len(q), _np_ptr(w),
                         cols_per_set, _np_ptr(flat), _dev_ptr(S_partial), _dev_ptr(S_total),
                         mode, _stream(stream)), "epsr_sq")


NOALLOC_MAX_ATOMS = 131072


def epsr_noalloc_scratch_bytes() -> int:
    return lib().epsr_noalloc_scratch_bytes()


def epsr_partial_gr_noalloc(system, hist, stream=None):
    """Pair histogram of one box with no device allocation (fixed library scratch); the
    coordinates and types are taken from host arrays of a synth.System-like object."""
    xyz = np.ascontiguousarray(system.xyz, np.int32)
    typ = np.ascontiguousarray(system.type, np.int32)
    n_pairs = system.n_types * (system.n_types + 1) // 2
    hp = _hist_ptr(hist, n_pairs * system.n_bins)
    _check(lib().epsr_partial_gr_noalloc(_np_ptr(xyz), _np_ptr(typ), xyz.shape[0], system.L_fx, 20,
                                         system.n_types, system.bin_p, system.bin_q, system.n_bins,
                                         hp, _stream(stream)), "epsr_partial_gr_noalloc")


class Refiner:
    """Owner of an epsr_refiner: the refinement loop (Sec. 2.2 items III-VI) on a one-box
    handle against measured S(Q) of n_data datasets (target device float [n_data][nQ])."""

    def __init__(self, box: Box, plan: SqPlan, target, w: np.ndarray, flat: np.ndarray, Q: np.ndarray,
                 moves_per_pass: int, seed: int = 1, move0: int = 0, accumulate: bool = False,
                 n_basis: int = 20, s_basis: float = 0.5, gamma: float = 0.0, alpha: float = 1.0,
                 stream=None):
        self.w = np.ascontiguousarray(np.atleast_2d(w), np.float64)
        self.flat = np.ascontiguousarray(np.atleast_1d(flat), np.float64)
        q = np.ascontiguousarray(Q, np.float32)
        self.n_data = self.w.shape[0]
        if target.numel() < self.n_data * len(q):
            raise ValueError("target: n_data x nQ elements needed")
        self.target, self.box, self.plan = target, box, plan
        self.n_basis = n_basis
        p = RefineParams(moves_per_pass, seed, move0, int(accumulate), n_basis, s_basis, gamma, alpha)
        h = C.c_void_p()
        _check(lib().epsr_refiner_create(box.h, plan.h, _dev_ptr(target), self.n_data, _np_ptr(self.w),
                                         _np_ptr(self.flat), _np_ptr(q), len(q), C.byref(p), _stream(stream),
                                         C.byref(h)), "epsr_refiner_create")
        self.h = h

    def step(self, log=None, stream=None) -> dict:
        r = RefineResult()
        _check(lib().epsr_refine_step(self.h, _dev_ptr(log), C.byref(r), _stream(stream)), "epsr_refine_step")
        return {f: getattr(r, f) for f, _ in RefineResult._fields_}

    def get(self, hist=None, g=None, S=None, dS=None, stream=None):
        """Copies the accumulated histogram, g, and S and Delta S of the last step into the given
        device tensors; returns the last fitted coefficients [n_pairs][n_basis]."""
        P = self.w.shape[1]
        Cb = np.zeros((P, self.n_basis), np.float64)
        _check(lib().epsr_refiner_get(self.h, _dev_ptr(hist), _dev_ptr(g), _dev_ptr(S), _dev_ptr(dS),
                                      _np_ptr(Cb), _stream(stream)), "epsr_refiner_get")
        return Cb

    def close(self):
        if getattr(self, "h", None):
            lib().epsr_refiner_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
