"""ctypes binding of libtvs.so (include/tvs.h).  Argument marshalling only:
every step of the computation runs in the library's CUDA kernels."""
from __future__ import annotations

import ctypes as C
import os
import re
import threading

import numpy as np

from . import _build

_lock = threading.Lock()
_lib = None

TVS_OK = 0
TVS_ERR_ARG = -1
TVS_ERR_OOM = -2
TVS_ERR_CUDA = -3
TVS_ERR_TIMEOUT = -4
TVS_ERR_STATE = -5
_ERRNAMES = {-1: "TVS_ERR_ARG", -2: "TVS_ERR_OOM", -3: "TVS_ERR_CUDA", -4: "TVS_ERR_TIMEOUT",
             -5: "TVS_ERR_STATE"}


class TvsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class DirectionInfo(C.Structure):
    _fields_ = [("frame", C.c_int32), ("m", C.c_int32), ("H", C.c_int32), ("W", C.c_int32),
                ("D", C.c_int32), ("R", C.c_int32), ("t_fx", C.c_uint64), ("t", C.c_double),
                ("g", C.c_double), ("K", C.c_int64)]


class TvsJob(C.Structure):
    _fields_ = [("d_dem", C.c_void_p), ("d_out", C.c_void_p), ("rows", C.c_int), ("cols", C.c_int),
                ("step_m", C.c_double), ("obs_height_m", C.c_double), ("n_sectors", C.c_int),
                ("max_range_m", C.c_double)]


class BatchInfo(C.Structure):
    _fields_ = [("jobs", C.c_int32), ("chunks", C.c_int32), ("kernels_per_launch", C.c_int32),
                ("pad_", C.c_int32), ("evals", C.c_double), ("scratch_bytes", C.c_double)]


class Tuning(C.Structure):
    _fields_ = [("small_pov_below_w", C.c_int32), ("sweep_max_warps", C.c_int32),
                ("unskew_ctas_per_sm", C.c_int32), ("p4_cost_pct", C.c_int32), ("prune", C.c_int32),
                ("fp32_decisions", C.c_int32)]


class ServerConfig(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("step_slot_bytes", C.c_size_t), ("step_evals", C.c_double),
                ("rate_hint", C.c_double), ("max_active", C.c_int32), ("policy", C.c_int32),
                ("lanes", C.c_int32), ("fail_after_steps", C.c_int32)]


class RequestInfo(C.Structure):
    _fields_ = [("state", C.c_int32), ("error", C.c_int32), ("steps", C.c_int32), ("n_sectors", C.c_int32),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_first", C.c_double),
                ("t_done", C.c_double), ("evals", C.c_double), ("message", C.c_char * 128)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64), ("steps", C.c_int64),
                ("kernels", C.c_int64), ("evals", C.c_double), ("arena_bytes", C.c_double),
                ("arena_peak_bytes", C.c_double), ("queued", C.c_int32), ("active", C.c_int32),
                ("max_step_jobs", C.c_int32), ("lanes", C.c_int32)]


POLICIES = {"deadline": 0, "fifo": 1, "srpt": 2}
REQUEST_STATES = {0: "queued", 1: "admitted", 2: "running", 3: "done", 4: "failed"}


class KernelStats(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("total_ms", C.c_double),
                ("units", C.c_double), ("unit", C.c_char * 16)]


def lib_path() -> str:
    return _build.LIB


def declared_functions() -> list[str]:
    """Names of the functions include/tvs.h declares."""
    with open(os.path.join(_build.INCLUDE, "tvs.h")) as f:
        text = f.read()
    return re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\**\s+\**\s*(tvs_[a-z_0-9]+)\s*\(", text, re.M)


def load(build_if_missing: bool = True) -> C.CDLL:
    """Load libtvs.so (building it first if allowed).  Raises if unavailable."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path) or not _build.up_to_date():
            if not build_if_missing:
                raise RuntimeError(f"{path} is missing or stale; build it with "
                                   "paper_2003_02200_gb300.build()")
            _build.build()
        lib = C.CDLL(path)
        vp, i32p, i64p = C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int64)
        sig = {
            "tvs_abi_version": ([], C.c_int),
            "tvs_create": ([C.POINTER(vp), C.c_int, C.c_size_t], C.c_int),
            "tvs_destroy": ([vp], None),
            "tvs_last_error": ([vp], C.c_char_p),
            "tvs_total_viewshed": ([vp, vp, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int,
                                    C.c_double, vp], C.c_int),
            "tvs_total_viewshed_device": ([vp, vp, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int,
                                           C.c_double, vp, vp], C.c_int),
            "tvs_total_viewshed_device_noalloc": ([vp, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int,
                                                   C.c_double, vp, vp], C.c_int),
            "tvs_total_viewshed_batch": ([vp, C.POINTER(TvsJob), C.c_int, vp], C.c_int),
            "tvs_batch_create": ([vp, C.POINTER(TvsJob), C.c_int, C.c_size_t, C.POINTER(vp)], C.c_int),
            "tvs_batch_launch": ([vp, vp], C.c_int),
            "tvs_batch_get_info": ([vp, C.POINTER(BatchInfo)], C.c_int),
            "tvs_batch_destroy": ([vp], None),
            "tvs_get_tuning": ([vp, C.POINTER(Tuning)], C.c_int),
            "tvs_set_tuning": ([vp, C.POINTER(Tuning)], C.c_int),
            "tvs_autotune": ([vp, C.POINTER(TvsJob), C.c_int, C.POINTER(Tuning), C.POINTER(C.c_double)], C.c_int),
            "tvs_direction": ([C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                               C.POINTER(DirectionInfo)], C.c_int),
            "tvs_count_evals": ([C.c_int, C.c_int, C.c_int, C.c_double, C.c_double], C.c_int64),
            "tvs_count_point_evals": ([C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, vp, C.c_int, C.c_int],
                                      C.c_int64),
            "tvs_debug_plan": ([vp, vp, vp, vp, vp, C.c_int, C.c_uint64, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp,
                                vp, C.c_int, i32p, i32p], C.c_int),
            "tvs_debug_rowmap": ([vp, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp, vp, vp, i32p], C.c_int),
            "tvs_debug_direction_cv": ([vp, vp, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int,
                                        C.c_double, C.c_int, vp, i32p, i32p], C.c_int),
            "tvs_debug_sweep_check": ([i32p, C.c_int], C.c_int),
            "tvs_debug_sweep_stats": ([C.POINTER(C.c_uint64), C.c_int], C.c_int),
            "tvs_viewshed_points": ([vp, vp, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, C.c_double, vp,
                                     C.c_int, C.c_int, vp, vp], C.c_int),
            "tvs_visibility_map": ([vp, vp, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, C.c_double, vp,
                                    C.c_int, vp, vp], C.c_int),
            "tvs_server_create": ([C.c_int, C.POINTER(ServerConfig), C.POINTER(vp)], C.c_int),
            "tvs_server_submit": ([vp, vp, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, C.c_double, vp,
                                   i64p], C.c_int),
            "tvs_server_wait": ([vp, C.c_int64, C.c_double], C.c_int),
            "tvs_server_query": ([vp, C.c_int64, C.POINTER(RequestInfo)], C.c_int),
            "tvs_server_get_stats": ([vp, C.POINTER(ServerStats)], C.c_int),
            "tvs_server_forget": ([vp, C.c_int64], C.c_int),
            "tvs_server_clock": ([vp], C.c_double),
            "tvs_server_destroy": ([vp], None),
            "tvs_profile_enable": ([vp, C.c_int], C.c_int),
            "tvs_profile_read": ([vp, C.POINTER(KernelStats), C.c_int, C.POINTER(C.c_int)], C.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(rc: int) -> None:
    if rc != TVS_OK:
        raise TvsError(rc, load().tvs_last_error(None).decode())


def _dem(dem) -> np.ndarray:
    a = np.ascontiguousarray(dem, dtype=np.float32)
    if a.ndim != 2:
        raise ValueError("dem must be a 2-D array")
    return a


def direction(n_sectors: int, k: int, rows: int, cols: int, step_m: float = 1.0,
              max_range_m: float = 0.0) -> dict:
    info = DirectionInfo()
    _check(load().tvs_direction(n_sectors, k, rows, cols, step_m, max_range_m, C.byref(info)))
    return {f: getattr(info, f) for f, _ in DirectionInfo._fields_}


def sweep_check(clear: bool = True) -> list[int]:
    """tvs_debug_sweep_check: the sweep's first out-of-range index on the
    current device as [code, index, bound, CTA] (all zero when none)."""
    out = (C.c_int32 * 4)()
    _check(load().tvs_debug_sweep_check(out, int(clear)))
    return list(out)


def sweep_stats(clear: bool = True) -> dict:
    """tvs_debug_sweep_stats: event counts of the certified sweep on the
    current device (exact walks, FP64 walks, warp cycles in exact walks and
    in the sweep)."""
    out = (C.c_uint64 * 4)()
    _check(load().tvs_debug_sweep_stats(out, int(clear)))
    return {"exact_walks": int(out[0]), "fp64_walks": int(out[1]), "exact_cycles": int(out[2]),
            "sweep_cycles": int(out[3])}


def count_evals(rows: int, cols: int, n_sectors: int, step_m: float = 1.0, max_range_m: float = 0.0) -> int:
    E = load().tvs_count_evals(rows, cols, n_sectors, step_m, max_range_m)
    if E < 0:
        _check(int(E))
    return int(E)


def debug_plan(jobs, budget_bytes: int, num_sms: int = 152, smem_optin: int = 0, prune: int = 1,
               fp32_decisions: int = 0):
    """tvs_debug_plan: the batch planner run on the host (no GPU) for jobs
    given as (rows, cols, n_sectors, step_m, max_range_m) tuples; returns
    the job, direction and chunk of every planned instance in launch order."""
    J = list(jobs)
    rows = np.array([j[0] for j in J], np.int32)
    cols = np.array([j[1] for j in J], np.int32)
    nsec = np.array([j[2] for j in J], np.int32)
    step = np.array([j[3] for j in J], np.float64)
    rng = np.array([j[4] for j in J], np.float64)
    cap = int(nsec.sum())
    ij, ik, ic = (np.zeros(max(cap, 1), np.int32) for _ in range(3))
    ninst, nchunks = C.c_int32(0), C.c_int32(0)
    _check(load().tvs_debug_plan(rows.ctypes.data, cols.ctypes.data, nsec.ctypes.data, step.ctypes.data,
                                 rng.ctypes.data, len(J), int(budget_bytes), num_sms, smem_optin, prune,
                                 fp32_decisions, ij.ctypes.data, ik.ctypes.data, ic.ctypes.data, cap,
                                 C.byref(ninst), C.byref(nchunks)))
    n = ninst.value
    return ij[:n].copy(), ik[:n].copy(), ic[:n].copy()


def count_point_evals(rows: int, cols: int, n_sectors: int, povs, step_m: float = 1.0, max_range_m: float = 0.0,
                      mode: str = "sdem") -> int:
    """tvs_count_point_evals: targets visited by tvs_viewshed_points."""
    p = np.ascontiguousarray(povs, dtype=np.int32).reshape(-1, 2)
    E = load().tvs_count_point_evals(rows, cols, n_sectors, step_m, max_range_m, p.ctypes.data, len(p),
                                     {"sdem": 0, "direct": 1}[mode])
    if E < 0:
        _check(int(E))
    return int(E)


def total_viewshed_device_noalloc(dem, step_m: float, obs_height_m: float, n_sectors: int = 180,
                                  max_range_m: float = 0.0, out=None, stream=None):
    """tvs_total_viewshed_device_noalloc on torch CUDA tensors of the current
    device: no handle, no device allocation by the library (its scratch is a
    fixed 64 MiB device array).  `out` must be given by callers that cannot
    allocate; when omitted it is created here with torch."""
    import torch
    if not (isinstance(dem, torch.Tensor) and dem.is_cuda and dem.dtype == torch.float32
            and dem.dim() == 2 and dem.is_contiguous()):
        raise ValueError("dem must be a contiguous 2-D float32 CUDA tensor")
    if out is None:
        out = torch.empty_like(dem)
    if out.shape != dem.shape or out.dtype != torch.float32 or not out.is_contiguous() or not out.is_cuda:
        raise ValueError("out must be a contiguous float32 CUDA tensor shaped like dem")
    if stream is None:
        stream = torch.cuda.current_stream(dem.device)
    _check(load().tvs_total_viewshed_device_noalloc(dem.data_ptr(), dem.shape[0], dem.shape[1], step_m,
                                                    obs_height_m, n_sectors, max_range_m, out.data_ptr(),
                                                    stream.cuda_stream))
    return out


def _job_array(jobs):
    """jobs: sequence of dicts with torch CUDA tensors dem, out and step_m,
    obs_height_m, n_sectors, max_range_m (defaults 180 directions, unlimited)."""
    import torch
    arr = (TvsJob * len(jobs))()
    for i, j in enumerate(jobs):
        dem, out = j["dem"], j["out"]
        for t in (dem, out):
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.dim() == 2
                    and t.is_contiguous()):
                raise ValueError(f"job {i}: dem and out must be contiguous 2-D float32 CUDA tensors")
        if out.shape != dem.shape:
            raise ValueError(f"job {i}: out must be shaped like dem")
        arr[i] = TvsJob(dem.data_ptr(), out.data_ptr(), dem.shape[0], dem.shape[1], float(j["step_m"]),
                        float(j["obs_height_m"]), int(j.get("n_sectors", 180)), float(j.get("max_range_m", 0.0)))
    return arr


class Batch:
    """A prepared batch (tvs_batch_create): fixed jobs, own scratch, launch
    sequence captured once in a CUDA graph and replayed by launch()."""

    def __init__(self, ctx: "Context", jobs, hbm_budget_bytes: int = 0):
        self._lib = load()
        self._jobs = list(jobs)          # keeps the tensors alive
        arr = _job_array(self._jobs)
        h = C.c_void_p()
        _check(self._lib.tvs_batch_create(ctx.handle, arr, len(arr), hbm_budget_bytes, C.byref(h)))
        self._b = h

    def launch(self, stream=None) -> None:
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        _check(self._lib.tvs_batch_launch(self._b, stream.cuda_stream))

    def info(self) -> dict:
        i = BatchInfo()
        _check(self._lib.tvs_batch_get_info(self._b, C.byref(i)))
        return {f: getattr(i, f) for f, _ in BatchInfo._fields_ if f != "pad_"}

    def close(self) -> None:
        if getattr(self, "_b", None):
            self._lib.tvs_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """A library handle bound to one CUDA device (tvs_create / tvs_destroy)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self._lib = load()
        h = C.c_void_p()
        _check(self._lib.tvs_create(C.byref(h), device, hbm_budget_bytes))
        self._h = h
        self.device = device

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.tvs_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self) -> C.c_void_p:
        if not self._h:
            raise RuntimeError("context is closed")
        return self._h

    def total_viewshed(self, dem, step_m: float, obs_height_m: float, n_sectors: int = 180,
                       max_range_m: float = 0.0, out: np.ndarray | None = None) -> np.ndarray:
        """tvs_total_viewshed on host arrays: returns the visible area (m^2) per cell."""
        a = _dem(dem)
        if out is None:
            out = np.empty_like(a)
        if out.shape != a.shape or out.dtype != np.float32 or not out.flags.c_contiguous:
            raise ValueError("out must be a C-contiguous float32 array shaped like dem")
        _check(self._lib.tvs_total_viewshed(self.handle, a.ctypes.data, a.shape[0], a.shape[1], step_m,
                                            obs_height_m, n_sectors, max_range_m, out.ctypes.data))
        return out

    def total_viewshed_device(self, dem, step_m: float, obs_height_m: float, n_sectors: int = 180,
                              max_range_m: float = 0.0, out=None, stream=None):
        """tvs_total_viewshed_device on torch CUDA tensors, ordered on `stream`
        (default: torch's current stream).  Returns `out`."""
        import torch
        if not (isinstance(dem, torch.Tensor) and dem.is_cuda and dem.dtype == torch.float32
                and dem.dim() == 2 and dem.is_contiguous()):
            raise ValueError("dem must be a contiguous 2-D float32 CUDA tensor")
        if out is None:
            out = torch.empty_like(dem)
        if out.shape != dem.shape or out.dtype != torch.float32 or not out.is_contiguous() or not out.is_cuda:
            raise ValueError("out must be a contiguous float32 CUDA tensor shaped like dem")
        if stream is None:
            stream = torch.cuda.current_stream(dem.device)
        _check(self._lib.tvs_total_viewshed_device(self.handle, dem.data_ptr(), dem.shape[0], dem.shape[1],
                                                   step_m, obs_height_m, n_sectors, max_range_m,
                                                   out.data_ptr(), stream.cuda_stream))
        return out

    def total_viewshed_batch(self, jobs, stream=None) -> None:
        """tvs_total_viewshed_batch: jobs as for Batch; results land in each job's out."""
        import torch
        arr = _job_array(jobs)
        if stream is None:
            stream = torch.cuda.current_stream()
        _check(self._lib.tvs_total_viewshed_batch(self.handle, arr, len(arr), stream.cuda_stream))

    def viewshed_points(self, dem, step_m: float, obs_height_m: float, n_sectors: int, max_range_m: float,
                        povs, mode: str = "sdem", out=None, stream=None):
        """tvs_viewshed_points: visible area (m^2) of each POV (row, col) of
        `povs` on a torch CUDA DEM; mode "sdem" (the total viewshed map's value
        at the cell) or "direct" (Alg. 1-3, lines through the cell itself).
        Returns a float32 CUDA tensor of len(povs) areas."""
        import torch
        if not (isinstance(dem, torch.Tensor) and dem.is_cuda and dem.dtype == torch.float32
                and dem.dim() == 2 and dem.is_contiguous()):
            raise ValueError("dem must be a contiguous 2-D float32 CUDA tensor")
        p = np.ascontiguousarray(povs, dtype=np.int32).reshape(-1, 2)
        if out is None:
            out = torch.empty(len(p), dtype=torch.float32, device=dem.device)
        if stream is None:
            stream = torch.cuda.current_stream(dem.device)
        m = {"sdem": 0, "direct": 1}[mode]
        _check(self._lib.tvs_viewshed_points(self.handle, dem.data_ptr(), dem.shape[0], dem.shape[1], step_m,
                                             obs_height_m, n_sectors, max_range_m, p.ctypes.data, len(p), m,
                                             out.data_ptr(), stream.cuda_stream))
        return out

    def visibility_map(self, dem, step_m: float, obs_height_m: float, n_sectors: int, max_range_m: float, povs,
                       out=None, stream=None):
        """tvs_visibility_map: int32 CUDA map of how many of the POVs (row, col)
        see each cell of the torch CUDA DEM."""
        import torch
        if not (isinstance(dem, torch.Tensor) and dem.is_cuda and dem.dtype == torch.float32
                and dem.dim() == 2 and dem.is_contiguous()):
            raise ValueError("dem must be a contiguous 2-D float32 CUDA tensor")
        p = np.ascontiguousarray(povs, dtype=np.int32).reshape(-1, 2)
        if out is None:
            out = torch.empty(dem.shape, dtype=torch.int32, device=dem.device)
        if stream is None:
            stream = torch.cuda.current_stream(dem.device)
        _check(self._lib.tvs_visibility_map(self.handle, dem.data_ptr(), dem.shape[0], dem.shape[1], step_m,
                                            obs_height_m, n_sectors, max_range_m, p.ctypes.data, len(p),
                                            out.data_ptr(), stream.cuda_stream))
        return out

    def get_tuning(self) -> dict:
        t = Tuning()
        _check(self._lib.tvs_get_tuning(self.handle, C.byref(t)))
        return {f: getattr(t, f) for f, _ in Tuning._fields_ if f != "pad_"}

    def set_tuning(self, **kw) -> None:
        cur = self.get_tuning()
        cur.update(kw)
        t = Tuning(cur["small_pov_below_w"], cur["sweep_max_warps"], cur["unskew_ctas_per_sm"], cur["p4_cost_pct"],
                   int(cur["prune"]), int(cur["fp32_decisions"]))
        _check(self._lib.tvs_set_tuning(self.handle, C.byref(t)))

    def autotune(self, jobs) -> tuple[dict, float]:
        """tvs_autotune on the given jobs; returns (best tuning, best batch ms)."""
        arr = _job_array(jobs)
        t = Tuning()
        ms = C.c_double(0.0)
        _check(self._lib.tvs_autotune(self.handle, arr, len(arr), C.byref(t), C.byref(ms)))
        return {f: getattr(t, f) for f, _ in Tuning._fields_ if f != "pad_"}, ms.value

    def prepare_batch(self, jobs, hbm_budget_bytes: int = 0) -> Batch:
        return Batch(self, jobs, hbm_budget_bytes)

    def debug_rowmap(self, rows: int, cols: int, n_sectors: int, k: int) -> dict:
        big = max(rows, cols)
        dest = np.empty(big, np.int32)
        frac = np.empty(big, np.uint32)
        jlo = np.empty(rows + cols, np.int32)
        jhi = np.empty(rows + cols, np.int32)
        R = C.c_int32(0)
        _check(self._lib.tvs_debug_rowmap(self.handle, rows, cols, n_sectors, k, dest.ctypes.data,
                                          frac.ctypes.data, jlo.ctypes.data, jhi.ctypes.data, C.byref(R)))
        W = direction(n_sectors, k, rows, cols)["W"]
        return dict(dest=dest[:W], frac=frac[:W], jlo=jlo[: R.value], jhi=jhi[: R.value], R=R.value)

    def debug_direction_cv(self, dem, step_m: float, obs_height_m: float, n_sectors: int,
                           max_range_m: float, k: int) -> np.ndarray:
        a = _dem(dem)
        rows, cols = a.shape
        buf = np.empty((rows + cols) * max(rows, cols), np.int32)
        R = C.c_int32(0)
        W = C.c_int32(0)
        _check(self._lib.tvs_debug_direction_cv(self.handle, a.ctypes.data, rows, cols, step_m, obs_height_m,
                                                n_sectors, max_range_m, k, buf.ctypes.data, C.byref(R),
                                                C.byref(W)))
        return buf[: R.value * W.value].reshape(R.value, W.value)

    def profile(self, on: bool) -> None:
        _check(self._lib.tvs_profile_enable(self.handle, 1 if on else 0))

    def profile_read(self) -> dict:
        arr = (KernelStats * 16)()
        cnt = C.c_int(0)
        _check(self._lib.tvs_profile_read(self.handle, arr, 16, C.byref(cnt)))
        return {arr[i].name.decode(): dict(launches=arr[i].launches, total_ms=arr[i].total_ms,
                                           units=arr[i].units, unit=arr[i].unit.decode())
                for i in range(cnt.value)}


class Server:
    """A request server (tvs_server_create): requests on host arrays are
    submitted as they arrive, admitted by the server's HBM budget and run in
    shared GPU steps (continuous batching).  submit() returns a ticket at once;
    wait() returns the finished visible-area map.  The arrays passed to
    submit() are kept alive here until their request finishes; page-locked
    arrays (e.g. numpy views of pinned torch tensors) make the copies
    asynchronous."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, step_slot_bytes: int = 0,
                 step_evals: float = 0.0, rate_hint: float = 0.0, max_active: int = 0, policy: str = "deadline",
                 lanes: int = 0, fail_after_steps: int = 0):
        self._lib = load()
        if policy not in POLICIES:
            raise ValueError(f"policy must be one of {sorted(POLICIES)}")
        cfg = ServerConfig(hbm_budget_bytes, step_slot_bytes, step_evals, rate_hint, max_active, POLICIES[policy],
                           lanes, fail_after_steps)
        h = C.c_void_p()
        _check(self._lib.tvs_server_create(device, C.byref(cfg), C.byref(h)))
        self._s = h
        self._live: dict[int, tuple[np.ndarray, np.ndarray]] = {}
        self._mu = threading.Lock()

    @property
    def handle(self) -> C.c_void_p:
        if not self._s:
            raise RuntimeError("server is closed")
        return self._s

    def submit(self, dem, step_m: float, obs_height_m: float, n_sectors: int = 180, max_range_m: float = 0.0,
               out: np.ndarray | None = None) -> int:
        a = _dem(dem)
        if out is None:
            out = np.empty_like(a)
        if out.shape != a.shape or out.dtype != np.float32 or not out.flags.c_contiguous:
            raise ValueError("out must be a C-contiguous float32 array shaped like dem")
        t = C.c_int64(0)
        _check(self._lib.tvs_server_submit(self.handle, a.ctypes.data, a.shape[0], a.shape[1], step_m, obs_height_m,
                                           n_sectors, max_range_m, out.ctypes.data, C.byref(t)))
        with self._mu:
            self._live[t.value] = (a, out)
        return t.value

    def wait(self, ticket: int, timeout: float = -1.0) -> np.ndarray:
        """Block until the request finishes; returns its output (raises
        TvsError on failure or timeout)."""
        _check(self._lib.tvs_server_wait(self.handle, ticket, timeout))
        with self._mu:
            _, out = self._live.pop(ticket)
        return out

    def query(self, ticket: int) -> dict:
        i = RequestInfo()
        _check(self._lib.tvs_server_query(self.handle, ticket, C.byref(i)))
        d = {f: getattr(i, f) for f, _ in RequestInfo._fields_}
        d["message"] = i.message.decode()
        d["state_name"] = REQUEST_STATES.get(i.state, str(i.state))
        return d

    def forget(self, ticket: int) -> None:
        """Drop the record of a finished request (tvs_server_forget)."""
        _check(self._lib.tvs_server_forget(self.handle, ticket))
        with self._mu:
            self._live.pop(ticket, None)

    def stats(self) -> dict:
        st = ServerStats()
        _check(self._lib.tvs_server_get_stats(self.handle, C.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def clock(self) -> float:
        return float(self._lib.tvs_server_clock(self.handle))

    def close(self) -> None:
        if getattr(self, "_s", None):
            self._lib.tvs_server_destroy(self._s)
            self._s = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
