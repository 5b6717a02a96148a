"""convtune — auto-tuned direct 2D correlation for GB300, Python binding.

A thin ctypes layer over ``libconvtune.so`` (``include/convtune.h``): it only
marshals arguments.  Every step of the correlation runs in the library's CUDA
kernels; PyTorch supplies device memory and streams.  There is no CPU
fallback: if the library is missing or cannot load, every call raises.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libconvtune.so")

CT_OK = 0
STATUS = {0: "CT_OK", -1: "CT_ERR_INVALID_ARG", -2: "CT_ERR_INVALID_CONFIG", -3: "CT_ERR_COMPILE",
          -4: "CT_ERR_LAUNCH", -5: "CT_ERR_CUDA", -6: "CT_ERR_OOM", -7: "CT_ERR_TIMEOUT", -8: "CT_ERR_UNSUPPORTED"}
CT_F32, CT_BF16 = 0, 1
STRATEGIES = {"brute": 0, "random": 1, "anneal": 2}
MAX_FILTER = 32

i32, i64, u64, dbl, vp, cp = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double,
                              ctypes.c_void_p, ctypes.c_char_p)


class CTError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Problem(ctypes.Structure):
    _fields_ = [("out_w", i32), ("out_h", i32), ("filter_w", i32), ("filter_h", i32),
                ("in_pitch", i64), ("out_pitch", i64), ("dtype", i32), ("reserved", i32)]


class Config(ctypes.Structure):
    """A point of the search space (the first six fields) plus four forms
    of the variant: ``persist`` (0: one block per tile, 1: persistent grid),
    ``taps`` (0: taps in the parameter block, 1: compiled into the variant),
    ``fma2`` (1: paired multiply-adds over pairs of output rows) and ``shfl``
    (1: window values from neighbouring lanes by warp shuffles)."""
    _fields_ = [("block_x", i32), ("block_y", i32), ("tile_x", i32), ("tile_y", i32),
                ("use_smem", i32), ("unroll", i32), ("persist", i32), ("taps", i32), ("fma2", i32),
                ("shfl", i32)]
    PARAMS = ("block_x", "block_y", "tile_x", "tile_y", "use_smem", "unroll", "persist", "taps", "fma2", "shfl")

    def as_dict(self):
        return {k: int(getattr(self, k)) for k in self.PARAMS}

    def as_tuple(self):
        return tuple(int(getattr(self, k)) for k in self.PARAMS)

    def space_tuple(self):
        """The six search-space parameters (without the grid choice)."""
        return self.as_tuple()[:6]

    def __repr__(self):
        return "Config(%s)" % ", ".join(f"{k}={v}" for k, v in self.as_dict().items())

    def __eq__(self, other):
        return isinstance(other, Config) and self.as_tuple() == other.as_tuple()

    def __hash__(self):
        return hash(self.as_tuple())


class VariantInfo(ctypes.Structure):
    _fields_ = [("regs", i32), ("spill_bytes", i32), ("smem_bytes", i32), ("cubin_bytes", i32),
                ("compile_ms", dbl), ("from_cache", i32), ("reserved", i32)]


class DeviceInfo(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 128), ("sm_count", i32), ("cc_major", i32), ("cc_minor", i32),
                ("smem_optin_bytes", i32), ("l2_bytes", i32), ("clock_max_khz", i32), ("reserved", i32)]


class TuneOpts(ctypes.Structure):
    _fields_ = [("seed", u64), ("sample_fraction", dbl), ("max_evals", i32), ("repeats", i32),
                ("warmup", i32), ("flush_l2", i32), ("compile_threads", i32), ("graph_below_us", i32),
                ("anneal_chains", i32), ("reserved", i32), ("cache_dir", cp), ("resume_path", cp),
                ("trace_path", cp), ("grid_modes", i32), ("remeasure_top", i32), ("remeasure_repeats", i32),
                ("taps_imm", i32), ("remeasure_forms", i32), ("sweep_fma2", i32)]


class Row(ctypes.Structure):
    _fields_ = [("cfg", Config), ("index", i64), ("status", i32), ("n", i32), ("t_med_ms", dbl),
                ("t_min_ms", dbl), ("t_std_ms", dbl), ("gflops", dbl), ("regs", i32), ("spill_bytes", i32),
                ("smem_bytes", i32), ("eval_order", i32), ("compile_ms", dbl), ("t_tiles_ms", dbl),
                ("t_persist_ms", dbl), ("t_remeasured_ms", dbl), ("sm_mhz", i32), ("reserved", i32)]


class TableInfo(ctypes.Structure):
    _fields_ = [("strategy", i32), ("n_rows", i32), ("n_valid_space", i64), ("best_row", i64),
                ("wall_ms", dbl), ("compile_wall_ms", dbl), ("compile_cpu_ms", dbl), ("bench_ms", dbl),
                ("remeasure_ms", dbl), ("remeasured", i32), ("sm_mhz_median", i32)]


class BatchItem(ctypes.Structure):
    _fields_ = [("d_image", vp), ("d_out", vp), ("h_filter", vp), ("out_w", i32), ("out_h", i32),
                ("filter_w", i32), ("filter_h", i32), ("in_pitch", i64), ("out_pitch", i64)]


class BucketConfig(ctypes.Structure):
    _fields_ = [("block_x", i32), ("block_y", i32), ("tile_x", i32), ("tile_y", i32), ("unroll", i32),
                ("fma2", i32)]


class BatchOpts(ctypes.Structure):
    _fields_ = [("dtype", i32), ("threads", i32), ("tune", i32), ("objective", i32), ("side_split", i32),
                ("blocks_per_sm", i32), ("max_tune_items", i32), ("solo_wave_pct", i32), ("solo_evals", i32),
                ("solo_branches", i32), ("bucket_forms", i32), ("persistent_layout", i32), ("work_order", i32),
                ("min_blocks_per_sm", i32)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("n_items", i32), ("n_buckets", i32), ("n_work", i64), ("grid", i32), ("threads", i32),
                ("smem_bytes", i32), ("regs", i32), ("plan_ms", dbl), ("tune_ms", dbl), ("compile_cpu_ms", dbl),
                ("n_solo", i32), ("n_solo_fma2", i32), ("persistent_beside", i32), ("work_interleaved", i32)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", i64), ("dtype", i32), ("max_batch", i32), ("max_launches", i32),
                ("max_wait_us", i32), ("tune", i32), ("filter_min", i32), ("filter_max", i32), ("reserved", i32),
                ("staging_bytes", i64)]


class Request(ctypes.Structure):
    _fields_ = [("h_image", vp), ("image_id", u64), ("h_out", vp), ("h_filter", vp), ("out_w", i32),
                ("out_h", i32), ("filter_w", i32), ("filter_h", i32), ("in_pitch", i64), ("out_pitch", i64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", i64), ("completed", i64), ("failed", i64), ("launches", i64), ("mean_batch", dbl),
                ("p50_ms", dbl), ("p99_ms", dbl), ("mean_ms", dbl), ("max_ms", dbl), ("wall_s", dbl),
                ("req_per_s", dbl), ("gflops", dbl), ("peak_mem_bytes", i64), ("kernel_busy_s", dbl),
                ("kernel_busy_frac", dbl)]


class ServerRunOpts(ctypes.Structure):
    _fields_ = [("n", i64), ("requests", ctypes.c_void_p), ("arrival_s", ctypes.c_void_p), ("max_in_flight", i32),
                ("reserved", i32), ("timeout_us", i64), ("latency_ms", ctypes.c_void_p)]


class Analysis(ctypes.Structure):
    _fields_ = [("n_valid", i64), ("n_minima", i64), ("best_index", i64), ("p_max", dbl), ("p_median", dbl),
                ("impact", dbl), ("tuned_vs_median", dbl), ("frac_within_10pct", dbl), ("quantiles", dbl * 7),
                ("n_p", i32), ("reserved", i32), ("p", dbl * 16), ("cp", dbl * 16)]


P = ctypes.POINTER
_SIGS = {
    "ct_version": (cp, []),
    "ct_last_error": (cp, []),
    "ct_device_query": (i32, [P(DeviceInfo)]),
    "ct_set_cache_dir": (i32, [cp]),
    "ct_clear_cache": (i32, []),
    "ct_default_config": (i32, [P(Problem), P(Config)]),
    "ct_check_config": (i32, [P(Problem), P(Config), i32]),
    "ct_compile": (i32, [P(Problem), P(Config), P(VariantInfo)]),
    "ct_compile_filter": (i32, [P(Problem), P(Config), vp, P(VariantInfo)]),
    "ct_device_check": (i32, [i32]),
    "ct_conv2d": (i32, [P(Problem), P(Config), vp, vp, vp, vp]),
    "ct_conv2d_host": (i32, [P(Problem), P(Config), vp, vp, vp, vp, vp, vp]),
    "ct_conv2d_host_pitched": (i32, [P(Problem), P(Config), vp, i64, vp, vp, i64, vp, vp, vp]),
    "ct_conv2d_host_async": (i32, [P(Problem), P(Config), vp, i64, vp, vp, i64, vp, vp, vp, vp]),
    "ct_space_builtin": (i32, [cp, P(vp)]),
    "ct_space_from_json": (i32, [cp, P(vp)]),
    "ct_space_free": (None, [vp]),
    "ct_space_count": (i32, [vp, P(Problem), i32, P(i64), P(i64)]),
    "ct_space_enumerate": (i32, [vp, P(Problem), i32, P(Config), P(i64), i64, P(i64)]),
    "ct_tune": (i32, [P(Problem), vp, i32, P(TuneOpts), vp, vp, vp, P(Config), P(vp)]),
    "ct_tune_replay": (i32, [P(Problem), vp, i32, P(TuneOpts), P(dbl), i64, P(Config), P(vp)]),
    "ct_table_size": (i64, [vp]),
    "ct_table_row": (i32, [vp, i64, P(Row)]),
    "ct_table_info_get": (i32, [vp, P(TableInfo)]),
    "ct_table_write": (i32, [vp, cp]),
    "ct_table_free": (None, [vp]),
    "ct_table_analyze": (i32, [vp, vp, dbl, P(dbl), i32, P(Analysis)]),
    "ct_batch_create": (i32, [P(BatchItem), i32, P(BatchOpts), P(vp)]),
    "ct_batch_run": (i32, [vp, vp]),
    "ct_batch_check": (i32, [vp]),
    "ct_batch_info_get": (i32, [vp, P(BatchInfo)]),
    "ct_batch_bucket": (i32, [vp, i32, P(i32), P(i32), P(i32), P(BucketConfig), P(dbl)]),
    "ct_batch_item_bucket": (i32, [vp, i32]),
    "ct_batch_free": (None, [vp]),
    "ct_batch_run_noalloc": (i32, [P(BatchItem), i32, i32, vp]),
    "ct_server_create": (i32, [P(ServerOpts), P(vp)]),
    "ct_server_image_register": (i32, [vp, vp, i32, i32, i64, P(u64)]),
    "ct_server_image_release": (i32, [vp, u64]),
    "ct_server_submit": (i32, [vp, P(Request), P(u64)]),
    "ct_server_wait": (i32, [vp, u64, i64, P(dbl)]),
    "ct_server_drain": (i32, [vp, i64]),
    "ct_server_stats_get": (i32, [vp, P(ServerStats)]),
    "ct_server_stats_reset": (i32, [vp]),
    "ct_server_run": (i32, [vp, P(ServerRunOpts), P(ServerStats)]),
    "ct_server_destroy": (None, [vp]),
}
EXPORTED = tuple(_SIGS)

_lock = threading.Lock()
_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"libconvtune.so is not built ({LIB_PATH}); run "
                                  "paper_2407_11488_gb300.build.build()")
            try:
                import torch  # noqa: F401  (shares its CUDA runtime with the library)
            except ImportError:
                pass
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def lib():
    """The loaded ctypes library (raises if it is missing)."""
    return _load()


def _check(status: int):
    if status != CT_OK:
        raise CTError(status, _load().ct_last_error().decode(errors="replace"))


def version() -> str:
    return _load().ct_version().decode()


def device_query() -> DeviceInfo:
    d = DeviceInfo()
    _check(_load().ct_device_query(ctypes.byref(d)))
    return d


def device_check(clear: bool = True):
    """Raises CTError(CT_ERR_TIMEOUT) when a ct_conv2d launch on the current
    device gave up waiting for its input copy (call after the launches have
    completed); clears the device's error word when ``clear``."""
    _check(_load().ct_device_check(1 if clear else 0))


def set_cache_dir(path):
    _check(_load().ct_set_cache_dir(path.encode() if path else None))


def clear_cache():
    _check(_load().ct_clear_cache())


def config(block_x=32, block_y=8, tile_x=1, tile_y=1, use_smem=0, unroll=0, persist=0, taps=0, fma2=0,
           shfl=0) -> Config:
    return Config(block_x, block_y, tile_x, tile_y, use_smem, unroll, persist, taps, fma2, shfl)


def default_config() -> Config:
    c = Config()
    _check(_load().ct_default_config(None, ctypes.byref(c)))
    return c


def round_up(v, m):
    return (v + m - 1) // m * m


def make_problem(out_w, out_h, filter_w, filter_h, *, in_pitch=None, out_pitch=None, dtype=CT_F32) -> Problem:
    if in_pitch is None:
        in_pitch = round_up(out_w + filter_w - 1, 8 if dtype == CT_BF16 else 4)
    if out_pitch is None:
        out_pitch = round_up(max(out_w, 1), 4)
    return Problem(out_w, out_h, filter_w, filter_h, in_pitch, out_pitch, dtype, 0)


def check_config(problem: Problem, cfg: Config, smem_limit: int = 0):
    _check(_load().ct_check_config(ctypes.byref(problem), ctypes.byref(cfg), smem_limit))


def compile_variant(problem: Problem, cfg: Config, filt=None) -> dict:
    """Compiles the variant (NVRTC → sm_103a cubin) without loading it; works
    without a GPU.  With ``filt`` (host filter) the variant ct_conv2d runs for
    that filter (filter-specific when cfg.taps = 1).  Returns the ptxas facts."""
    info = VariantInfo()
    if filt is None:
        _check(_load().ct_compile(ctypes.byref(problem), ctypes.byref(cfg), ctypes.byref(info)))
    else:
        fb = _filter_bytes(filt, problem.dtype)
        _check(_load().ct_compile_filter(ctypes.byref(problem), ctypes.byref(cfg), fb.ctypes.data_as(vp),
                                         ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in VariantInfo._fields_ if k != "reserved"}


# ------------------------------------------------------------ correlation ---
def _dtype_code(t):
    import torch
    if t.dtype == torch.float32:
        return CT_F32
    if t.dtype == torch.bfloat16:
        return CT_BF16
    raise TypeError(f"image dtype {t.dtype} is not float32 or bfloat16")


def _filter_bytes(filt, dtype):
    """Host copy of the filter as float32 (CT_F32) or raw bf16 bits (CT_BF16)."""
    import torch
    if isinstance(filt, torch.Tensor):
        f = filt.detach().cpu()
        if dtype == CT_BF16:
            if f.dtype != torch.bfloat16:
                raise TypeError("a bf16 problem needs a bfloat16 filter")
            arr = f.contiguous().view(torch.int16).numpy().view(np.uint16)
        else:
            arr = f.to(torch.float32).contiguous().numpy()
    else:
        arr = np.ascontiguousarray(filt, dtype=np.uint16 if dtype == CT_BF16 else np.float32)
    if arr.ndim != 2:
        raise ValueError("filter must be 2-D (filter_h, filter_w)")
    return np.ascontiguousarray(arr)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def problem_for(image, filt, in_w=None, out_pitch=None) -> Problem:
    """The Problem for an image tensor of shape (in_h, in_pitch) whose first
    ``in_w`` columns are valid (default: all of them) and a (fh, fw) filter."""
    fh, fw = int(filt.shape[0]), int(filt.shape[1])
    in_h, pitch = int(image.shape[0]), int(image.stride(0))
    if in_w is None:
        in_w = int(image.shape[1])
    out_w, out_h = in_w - fw + 1, in_h - fh + 1
    if out_w < 0 or out_h < 0:
        raise ValueError("filter larger than image")
    if out_pitch is None:
        out_pitch = round_up(max(out_w, 1), 4)
    return Problem(out_w, out_h, fw, fh, pitch, out_pitch, _dtype_code(image), 0)


def conv2d(image, filt, cfg: Config | None = None, *, in_w=None, out=None, stream=None):
    """Valid cross-correlation of a device image with a host filter.

    image: CUDA tensor (in_h, in_pitch), float32 or bfloat16, rows 16-byte
    aligned; filt: (fh, fw) host array/tensor; out: optional CUDA float32
    tensor (out_h, out_pitch).  Enqueued on ``stream`` (default: torch's
    current stream).  Returns the (out_h, out_w) view of the output."""
    import torch
    if not isinstance(image, torch.Tensor) or not image.is_cuda:
        raise TypeError("image must be a CUDA tensor")
    if image.stride(1) != 1:
        raise ValueError("image rows must be contiguous")
    p = problem_for(image, filt, in_w)
    fb = _filter_bytes(filt, p.dtype)
    if out is None:
        out = torch.empty((p.out_h, p.out_pitch), dtype=torch.float32, device=image.device)
    else:
        if out.dtype != torch.float32 or not out.is_cuda or out.stride(1) != 1:
            raise TypeError("out must be a CUDA float32 tensor with contiguous rows")
        p.out_pitch = out.stride(0)
        if out.shape[0] < p.out_h or out.shape[1] < p.out_w:
            raise ValueError("out is too small")
    cfg = cfg or default_config()
    _check(_load().ct_conv2d(ctypes.byref(p), ctypes.byref(cfg), ctypes.c_void_p(image.data_ptr()),
                             fb.ctypes.data_as(vp), ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out[:p.out_h, :p.out_w]


def conv2d_raw(problem: Problem, cfg: Config, d_image: int, h_filter: np.ndarray, d_out: int, stream: int = 0):
    """ct_conv2d on raw device addresses (for timing loops)."""
    _check(_load().ct_conv2d(ctypes.byref(problem), ctypes.byref(cfg), ctypes.c_void_p(d_image),
                             h_filter.ctypes.data_as(vp), ctypes.c_void_p(d_out), ctypes.c_void_p(stream)))


def conv2d_host(problem: Problem, cfg: Config, h_image, h_filter: np.ndarray, h_out, d_image_ws, d_out_ws,
                stream=None):
    """End-to-end: host image in, host output out (copies on the stream, then
    a synchronisation).  All arrays are torch tensors (host ones pinned)."""
    _check(_load().ct_conv2d_host(ctypes.byref(problem), ctypes.byref(cfg), ctypes.c_void_p(h_image.data_ptr()),
                                  h_filter.ctypes.data_as(vp), ctypes.c_void_p(h_out.data_ptr()),
                                  ctypes.c_void_p(d_image_ws.data_ptr()), ctypes.c_void_p(d_out_ws.data_ptr()),
                                  _stream_ptr(stream)))


def conv2d_host_pitched(problem: Problem, cfg: Config, h_image, h_in_pitch: int, h_filter: np.ndarray, h_out,
                        h_out_pitch: int, d_image_ws, d_out_ws, stream=None):
    """ct_conv2d_host with host rows of their own pitch (2D copies)."""
    _check(_load().ct_conv2d_host_pitched(ctypes.byref(problem), ctypes.byref(cfg), ctypes.c_void_p(h_image),
                                          h_in_pitch, h_filter.ctypes.data_as(vp), ctypes.c_void_p(h_out),
                                          h_out_pitch, ctypes.c_void_p(d_image_ws), ctypes.c_void_p(d_out_ws),
                                          _stream_ptr(stream)))


def conv2d_host_async(problem: Problem, cfg: Config, h_image, h_in_pitch: int, h_filter: np.ndarray, h_out,
                      h_out_pitch: int, d_image_ws, d_out_ws, done_event, stream=None):
    """ct_conv2d_host_async: enqueue, signal completion on done_event (a
    torch.cuda.Event); the caller keeps the buffers untouched until then."""
    import torch
    if done_event.cuda_event == 0:          # torch creates the event on its first record
        done_event.record(torch.cuda.current_stream())
    _check(_load().ct_conv2d_host_async(ctypes.byref(problem), ctypes.byref(cfg), ctypes.c_void_p(h_image),
                                        h_in_pitch, h_filter.ctypes.data_as(vp), ctypes.c_void_p(h_out), h_out_pitch,
                                        ctypes.c_void_p(d_image_ws), ctypes.c_void_p(d_out_ws), _stream_ptr(stream),
                                        ctypes.c_void_p(done_event.cuda_event)))


# ------------------------------------------------------------------ spaces ---
class Space:
    """A search space handle (built-in name or JSON text)."""

    def __init__(self, spec="small"):
        h = vp()
        if spec.lstrip().startswith("{"):
            _check(_load().ct_space_from_json(spec.encode(), ctypes.byref(h)))
        else:
            _check(_load().ct_space_builtin(spec.encode(), ctypes.byref(h)))
        self.handle = h
        self.spec = spec

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.ct_space_free(self.handle)
            self.handle = None

    def count(self, problem: Problem, smem_limit: int = 0):
        raw, valid = i64(), i64()
        _check(_load().ct_space_count(self.handle, ctypes.byref(problem), smem_limit, ctypes.byref(raw),
                                      ctypes.byref(valid)))
        return raw.value, valid.value

    def enumerate(self, problem: Problem, smem_limit: int = 0):
        n = i64()
        _check(_load().ct_space_enumerate(self.handle, ctypes.byref(problem), smem_limit, None, None, 0,
                                          ctypes.byref(n)))
        cfgs = (Config * n.value)()
        idx = (i64 * n.value)()
        _check(_load().ct_space_enumerate(self.handle, ctypes.byref(problem), smem_limit, cfgs, idx, n.value,
                                          ctypes.byref(n)))
        return [(int(idx[i]), cfgs[i]) for i in range(n.value)]


def _space(space):
    return space if isinstance(space, Space) else Space(space)


# ------------------------------------------------------------------ tuning ---
@dataclass
class Table:
    rows: list
    info: dict
    best: Config | None
    analysis: dict | None = None

    def valid(self):
        return [r for r in self.rows if r["status"] == 0 and math.isfinite(r["t_med_ms"])]


def _row_dict(r: Row) -> dict:
    d = {k: getattr(r, k) for k, _ in Row._fields_ if k not in ("cfg", "reserved")}
    d["cfg"] = Config(*r.cfg.as_tuple())
    d.update(r.cfg.as_dict())
    return d


P_VALUES = (0.0, 0.01, 0.02, 0.05, 0.10, 0.15)


def _analysis(t, space, flops):
    a = Analysis()
    pv = (dbl * len(P_VALUES))(*P_VALUES)
    if _load().ct_table_analyze(t, space.handle, flops, pv, len(P_VALUES), ctypes.byref(a)) != CT_OK:
        return None
    d = {k: getattr(a, k) for k in ("n_valid", "n_minima", "best_index", "p_max", "p_median", "impact",
                                     "tuned_vs_median", "frac_within_10pct")}
    d["quantiles"] = dict(zip((0, 10, 25, 50, 75, 90, 100), list(a.quantiles)))
    d["cp"] = {P_VALUES[k]: a.cp[k] for k in range(a.n_p)}
    return d


def _collect(t, best, write_path=None, space=None, flops=0.0) -> Table:
    L = _load()
    try:
        if write_path:
            _check(L.ct_table_write(t, write_path.encode()))
        info = TableInfo()
        _check(L.ct_table_info_get(t, ctypes.byref(info)))
        rows = []
        for i in range(L.ct_table_size(t)):
            r = Row()
            _check(L.ct_table_row(t, i, ctypes.byref(r)))
            rows.append(_row_dict(r))
        infod = {k: getattr(info, k) for k, _ in TableInfo._fields_}
        return Table(rows, infod, best, _analysis(t, space, flops) if space is not None else None)
    finally:
        L.ct_table_free(t)


def _opts(seed=0, sample_fraction=0.0, max_evals=0, repeats=0, warmup=0, flush_l2=False, compile_threads=0,
          graph_below_us=0, anneal_chains=0, cache_dir=None, resume_path=None, trace_path=None, grid_modes=0,
          remeasure_top=0, remeasure_repeats=0, taps_imm=0, remeasure_forms=0, sweep_fma2=0):
    return TuneOpts(seed, sample_fraction, max_evals, repeats, warmup, int(flush_l2), compile_threads,
                    graph_below_us, anneal_chains, 0, cache_dir.encode() if cache_dir else None,
                    resume_path.encode() if resume_path else None, trace_path.encode() if trace_path else None,
                    int(grid_modes), remeasure_top, remeasure_repeats, int(taps_imm), int(remeasure_forms),
                    int(sweep_fma2))


def tune(problem: Problem, space="small", strategy="brute", *, image=None, filt=None, out=None,
         write_path=None, **opts) -> Table:
    """ct_tune: compile, launch and time every configuration the strategy
    visits on the GPU; returns the timing table with its best config."""
    sp = _space(space)
    o = _opts(**opts)
    fb = _filter_bytes(filt, problem.dtype) if filt is not None else None
    best = Config()
    t = vp()
    st = _load().ct_tune(ctypes.byref(problem), sp.handle, STRATEGIES[strategy], ctypes.byref(o),
                         ctypes.c_void_p(image.data_ptr()) if image is not None else None,
                         fb.ctypes.data_as(vp) if fb is not None else None,
                         ctypes.c_void_p(out.data_ptr()) if out is not None else None,
                         ctypes.byref(best), ctypes.byref(t))
    if t.value:
        flops = 2.0 * problem.out_w * problem.out_h * problem.filter_w * problem.filter_h
        table = _collect(t, best if st == CT_OK else None, write_path, sp, flops)
        if st != CT_OK:
            raise CTError(st, _load().ct_last_error().decode(errors="replace"))
        return table
    _check(st)
    raise CTError(-5, "ct_tune returned no table")


def tune_replay(problem: Problem, space, strategy, times_ms, **opts) -> Table:
    """The strategies over a given landscape: times_ms[k] is the time of the
    configuration with canonical index k (NaN/<=0: failing)."""
    sp = _space(space)
    o = _opts(**opts)
    arr = np.ascontiguousarray(times_ms, dtype=np.float64)
    best = Config()
    t = vp()
    st = _load().ct_tune_replay(ctypes.byref(problem), sp.handle, STRATEGIES[strategy], ctypes.byref(o),
                                arr.ctypes.data_as(P(dbl)), len(arr), ctypes.byref(best), ctypes.byref(t))
    if t.value:
        flops = 2.0 * problem.out_w * problem.out_h * problem.filter_w * problem.filter_h
        return _collect(t, best if st == CT_OK else None, None, sp, flops)
    _check(st)
    raise CTError(-5, "ct_tune_replay returned no table")


# ------------------------------------------------------------------ batches ---
class Batch:
    """Many uneven correlations in one graph launch (ct_batch_*): a
    persistent launch over all problems, except those that fill at least
    ``solo_wave_pct`` percent of one wave of the GPU (0: 10; < 0: none),
    which run as their own launches of the single-problem kernel, spread over
    ``solo_branches`` parallel graph branches (0: 12).  ``bucket_forms``:
    the bucket tiles tried when tuning ("both", "scalar" or "paired"
    multiply-adds; with ``tune=False``, "paired" gives the default tile in the
    paired form).  ``persistent_layout``: where the persistent launch sits in
    the graph ("timed": both layouts timed, the faster kept; "after" the solo
    launches; "beside" them, on a branch of its own).  ``work_order``: the
    persistent launch's work list ("timed", "buckets": one bucket after
    another, "interleaved").  ``min_blocks_per_sm``: resident blocks per SM
    the persistent kernel is built for (0: 4).

    ``problems`` is a list of (image, filt, out, in_w): CUDA image tensor
    (in_h, in_pitch) with in_w valid columns, host filter (fh, fw), CUDA
    float32 output tensor (out_h >= rows, out_pitch).  The tensors must stay
    alive while the batch is used; filters are copied at creation."""

    def __init__(self, problems, *, dtype=None, threads=256, tune=True, objective="pp", side_split=512,
                 blocks_per_sm=0, max_tune_items=12, solo_wave_pct=0, solo_evals=0, solo_branches=0,
                 bucket_forms="both", persistent_layout="timed", work_order="timed", min_blocks_per_sm=0):
        import torch
        self._keep = []
        arr = (BatchItem * len(problems))()
        dt = None
        for k, (img, filt, out, in_w) in enumerate(problems):
            p = problem_for(img, filt, in_w)
            dt = p.dtype if dt is None else dt
            if p.dtype != dt:
                raise TypeError("all images of a batch share one dtype")
            fb = _filter_bytes(filt, p.dtype)
            if out.dtype != torch.float32 or not out.is_cuda:
                raise TypeError("outputs must be CUDA float32 tensors")
            self._keep += [img, out, fb]
            arr[k] = BatchItem(img.data_ptr(), out.data_ptr(), fb.ctypes.data, p.out_w, p.out_h, p.filter_w,
                               p.filter_h, p.in_pitch, out.stride(0))
        o = BatchOpts(dt if dtype is None else dtype, threads, int(tune), 1 if objective == "time" else 0,
                      side_split, blocks_per_sm, max_tune_items, solo_wave_pct, solo_evals, solo_branches,
                      {"both": 0, "scalar": 1, "paired": 2}[bucket_forms],
                      {"timed": 0, "after": 1, "beside": 2}[persistent_layout],
                      {"timed": 0, "buckets": 1, "interleaved": 2}[work_order], min_blocks_per_sm)
        h = vp()
        _check(_load().ct_batch_create(arr, len(problems), ctypes.byref(o), ctypes.byref(h)))
        self.handle = h
        self.n = len(problems)

    def run(self, stream=None):
        _check(_load().ct_batch_run(self.handle, _stream_ptr(stream)))

    def check(self):
        """Raises CTError(CT_ERR_TIMEOUT) when a block of an earlier run gave
        up waiting for its input copies; call after the runs completed."""
        _check(_load().ct_batch_check(self.handle))

    def info(self) -> dict:
        i = BatchInfo()
        _check(_load().ct_batch_info_get(self.handle, ctypes.byref(i)))
        return {k: getattr(i, k) for k, _ in BatchInfo._fields_}

    def buckets(self):
        res = []
        for k in range(self.info()["n_buckets"]):
            fw, fh, n = i32(), i32(), i32()
            c = BucketConfig()
            pp = dbl()
            _check(_load().ct_batch_bucket(self.handle, k, ctypes.byref(fw), ctypes.byref(fh), ctypes.byref(n),
                                           ctypes.byref(c), ctypes.byref(pp)))
            res.append({"filter": (fw.value, fh.value), "n_items": n.value, "pp": pp.value,
                        "config": {f: getattr(c, f) for f, _ in BucketConfig._fields_}})
        return res

    def item_bucket(self, i: int) -> int:
        return int(_load().ct_batch_item_bucket(self.handle, i))

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.ct_batch_free(self.handle)
            self.handle = None


# ------------------------------------------------------------------ serving ---
class Server:
    """Continuous-batching request server (ct_server_*).  Host buffers passed
    to submit() are kept referenced until the request is waited."""

    def __init__(self, mem_budget_bytes, *, dtype=CT_F32, max_batch=64, max_launches=3, max_wait_us=200,
                 tune=True, filter_min=3, filter_max=17, staging_bytes=0):
        o = ServerOpts(int(mem_budget_bytes), dtype, max_batch, max_launches, max_wait_us, int(tune), filter_min,
                       filter_max, 0, int(staging_bytes))
        h = vp()
        _check(_load().ct_server_create(ctypes.byref(o), ctypes.byref(h)))
        self.handle = h
        self.dtype = dtype
        self._refs = {}
        self._fcache = {}   # filter object id -> (filter, its bytes), for run() requests

    def register_image(self, h_image, in_w=None) -> int:
        """Uploads a host image tensor (in_h, in_pitch) that stays resident."""
        iid = u64()
        in_w = int(h_image.shape[1]) if in_w is None else in_w
        _check(_load().ct_server_image_register(self.handle, ctypes.c_void_p(h_image.data_ptr()), in_w,
                                                int(h_image.shape[0]), int(h_image.stride(0)), ctypes.byref(iid)))
        return iid.value

    def release_image(self, image_id: int):
        _check(_load().ct_server_image_release(self.handle, image_id))

    def submit(self, h_out, filt, out_w, out_h, *, h_image=None, image_id=0, in_pitch=None) -> int:
        fb = _filter_bytes(filt, self.dtype)
        fh, fw = fb.shape
        if in_pitch is None:
            in_pitch = int(h_image.stride(0)) if h_image is not None else 0
        rq = Request(ctypes.c_void_p(h_image.data_ptr()) if h_image is not None else None, image_id,
                     ctypes.c_void_p(h_out.data_ptr()), fb.ctypes.data_as(vp), out_w, out_h, fw, fh, in_pitch,
                     int(h_out.stride(0)))
        rid = u64()
        _check(_load().ct_server_submit(self.handle, ctypes.byref(rq), ctypes.byref(rid)))
        self._refs[rid.value] = (h_image, h_out, fb)
        return rid.value

    def wait(self, request_id: int, timeout_us: int = -1) -> float:
        lat = dbl()
        st = _load().ct_server_wait(self.handle, request_id, timeout_us, ctypes.byref(lat))
        if st != -7:
            self._refs.pop(request_id, None)
        _check(st)
        return lat.value

    def drain(self, timeout_us: int = -1):
        _check(_load().ct_server_drain(self.handle, timeout_us))

    def stats(self) -> dict:
        st = ServerStats()
        _check(_load().ct_server_stats_get(self.handle, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def reset_stats(self):
        _check(_load().ct_server_stats_reset(self.handle))

    def request(self, h_out, filt, out_w, out_h, *, h_image=None, image_id=0, in_pitch=None) -> Request:
        """A request record for run(); the filter bytes are kept alive by the server object."""
        key = id(filt)
        hit = self._fcache.get(key)
        if hit is None or hit[0] is not filt:
            hit = (filt, _filter_bytes(filt, self.dtype))
            self._fcache[key] = hit
        fb = hit[1]
        fh, fw = fb.shape
        if in_pitch is None:
            in_pitch = int(h_image.stride(0)) if h_image is not None else 0
        return Request(ctypes.c_void_p(h_image.data_ptr()) if h_image is not None else None, image_id,
                       ctypes.c_void_p(h_out.data_ptr()), fb.ctypes.data_as(vp), out_w, out_h, fw, fh, in_pitch,
                       int(h_out.stride(0)))

    def run(self, requests, *, arrival_s=None, max_in_flight=64, timeout_us=120_000_000):
        """ct_server_run: submit `requests` (a list of Request, or a ctypes array)
        from native threads, paced by arrival_s (seconds from the start) or
        closed loop; returns (stats dict, latencies in ms as a numpy array)."""
        n = len(requests)
        arr = requests if isinstance(requests, ctypes.Array) else (Request * n)(*requests)
        lat = np.full(n, np.nan)
        arrivals = None if arrival_s is None else np.ascontiguousarray(arrival_s, dtype=np.float64)
        o = ServerRunOpts(n, ctypes.cast(arr, vp), arrivals.ctypes.data if arrivals is not None else None,
                          max_in_flight, 0, timeout_us, lat.ctypes.data)
        st = ServerStats()
        _check(_load().ct_server_run(self.handle, ctypes.byref(o), ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}, lat

    def close(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.ct_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()
