"""GB300 (sm_103a) frequency-domain coherent beamformer.

Python binding of the C ABI declared in ``include/bf.h`` (``libbf.so``, built
in-tree by ``paper_1412_4907_gb300.build``).  The functions keep the C names
and only marshal arguments: every step of the computation runs in the CUDA
kernels of the library.  Device buffers are passed as integer addresses (for
example ``tensor.data_ptr()``) and streams as ``cudaStream_t`` integers.  If
the library is missing, importing the binding raises: there is no fallback.

``Plan`` wraps a plan with torch tensors for convenience (torch provides
device memory and streams only).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbf.so")

BF_OK, BF_ERR_ARG, BF_ERR_NOMEM, BF_ERR_CUDA, BF_ERR_TIMEOUT, BF_ERR_UNSUPPORTED, BF_ERR_STATE = range(7)
BF_C32, BF_C16F, BF_C16BF, BF_C8E4M3, BF_CI8, BF_CI4 = range(6)
BF_LAYOUT_CTN, BF_LAYOUT_NCT = 0, 1
BF_KERNEL_AUTO, BF_KERNEL_SIMT, BF_KERNEL_TC = 0, 1, 2

SAMPLE_BYTES = {BF_C32: 8, BF_C16F: 4, BF_C16BF: 4, BF_C8E4M3: 2, BF_CI8: 2, BF_CI4: 1}
STATUS_NAMES = {0: "BF_OK", 1: "BF_ERR_ARG", 2: "BF_ERR_NOMEM", 3: "BF_ERR_CUDA",
                4: "BF_ERR_TIMEOUT", 5: "BF_ERR_UNSUPPORTED", 6: "BF_ERR_STATE"}

# every entry point declared in include/bf.h, with its ctypes signature
_P, _I, _S = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t


class bf_completion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_longlong), ("config", ctypes.c_int), ("status", ctypes.c_int),
                ("n_windows", ctypes.c_int), ("step", ctypes.c_int), ("n_samp", ctypes.c_int),
                ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double), ("t_done", ctypes.c_double)]


class bf_server_counters(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong), ("steps", ctypes.c_longlong),
                ("max_jobs_per_step", ctypes.c_int), ("tile_t", ctypes.c_int), ("flops", ctypes.c_double),
                ("kernel_ms", ctypes.c_double), ("copy_in_ms", ctypes.c_double), ("copy_in_bytes", ctypes.c_double),
                ("arena_bytes", ctypes.c_size_t), ("arena_peak", ctypes.c_size_t)]

SIGNATURES = {
    "bf_plan_create": [ctypes.POINTER(_P), _I, _P, _P, _I, _P, _I, _P, _I, _I, _I, _P],
    "bf_weights": [_P, _P],
    "bf_execute": [_P, _P, _I, _P, _P],
    "bf_execute_complex": [_P, _P, _I, _P, _P],
    "bf_execute_incoherent": [_P, _P, _I, _P, _P],
    "bf_execute_host": [_P, _P, _I, _P],
    "bf_sync": [_P],
    "bf_destroy": [_P],
    "bf_last_error": [],
    "bf_plan_set_kernel": [_P, _I, _I],
    "bf_plan_set_input_order": [_P, _P],
    "bf_plan_set_tiles": [_P, _I, _I, _I],
    "bf_plan_set_weight_buffers": [_P, _I],
    "bf_plan_query_tiles": [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "bf_plan_query": [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_S)],
    "bf_export_weights": [_P, _P, _P],
    "bf_corner_turn": [_P, _I, _P, _I, _I, _I, _I, _P, _P],
    "bf_batch_create": [ctypes.POINTER(_P), _P, _I, _I],
    "bf_batch_set": [_P, _I, _P, _I, _P],
    "bf_batch_execute": [_P, _P],
    "bf_batch_capture": [_P, _P],
    "bf_batch_replay": [_P, _P],
    "bf_batch_sync": [_P],
    "bf_batch_query": [_P, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double)],
    "bf_batch_destroy": [_P],
    "bf_server_create": [ctypes.POINTER(_P), _P, _I, _S, _I, _I],
    "bf_server_submit": [_P, _I, _P, _I, _P, ctypes.POINTER(ctypes.c_longlong)],
    "bf_server_poll": [_P, ctypes.POINTER(bf_completion), _I, ctypes.POINTER(_I), _I],
    "bf_server_drain": [_P, _I],
    "bf_server_pause": [_P, _I],
    "bf_server_stats": [_P, ctypes.POINTER(bf_server_counters)],
    "bf_server_destroy": [_P],
    "bf_server_now": [],
    "bf_detect": [_P, _I, _I, _I, ctypes.c_float, _P, _P, _I, _P, _P],
    "bf_selftest_timeout": [ctypes.c_double, _P],
    "bf_measure_ffma": [ctypes.c_double, ctypes.POINTER(ctypes.c_double), _P],
    "bf_execute_nct_static": [_P, _P, _I, _P, _P],
}


class BFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run paper_1412_4907_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    for name, argtypes in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = argtypes
        fn.restype = {"bf_last_error": ctypes.c_char_p, "bf_server_now": ctypes.c_double}.get(name, ctypes.c_int)
    return lib


_lib = _load()


def _check(rc: int):
    if rc != BF_OK:
        raise BFError(rc, _lib.bf_last_error().decode())


def _host(a, dtype):
    if a is None:
        return None, None
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr, arr.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------- C-named thin wrappers
def bf_plan_create(pos_m, freqs_hz, dirs, dtype: int, t_int: int, layout: int = BF_LAYOUT_CTN,
                   mask=None, stream: int = 0) -> int:
    pos, pp = _host(pos_m, np.float64)
    fr, fp = _host(freqs_hz, np.float64)
    di, dp = _host(dirs, np.float64)
    mk, mp = _host(mask, np.uint8)
    plan = ctypes.c_void_p()
    _check(_lib.bf_plan_create(ctypes.byref(plan), pos.shape[0], pp, mp, fr.shape[0], fp,
                               di.shape[0], dp, dtype, t_int, layout, stream or None))
    return plan.value


def bf_weights(plan: int, dirs=None):
    di, dp = _host(dirs, np.float64)
    _check(_lib.bf_weights(plan, dp))


def bf_execute(plan: int, d_voltages: int, n_samp: int, d_power: int, stream: int = 0):
    _check(_lib.bf_execute(plan, d_voltages, n_samp, d_power, stream or None))


def bf_execute_complex(plan: int, d_voltages: int, n_samp: int, d_beams: int, stream: int = 0):
    _check(_lib.bf_execute_complex(plan, d_voltages, n_samp, d_beams, stream or None))


def bf_execute_incoherent(plan: int, d_voltages: int, n_samp: int, d_power: int, stream: int = 0):
    _check(_lib.bf_execute_incoherent(plan, d_voltages, n_samp, d_power, stream or None))


def bf_execute_host(plan: int, h_voltages: int, n_samp: int, h_power: int):
    _check(_lib.bf_execute_host(plan, h_voltages, n_samp, h_power))


def bf_execute_nct_static(plan: int, d_voltages: int, n_samp: int, d_power: int, stream: int = 0):
    _check(_lib.bf_execute_nct_static(plan, d_voltages, n_samp, d_power, stream or None))


def bf_sync(plan: int):
    _check(_lib.bf_sync(plan))


def bf_destroy(plan: int):
    _check(_lib.bf_destroy(plan))


def bf_last_error() -> str:
    return _lib.bf_last_error().decode()


def bf_plan_set_kernel(plan: int, kernel: int, tile_t: int = 0):
    _check(_lib.bf_plan_set_kernel(plan, kernel, tile_t))


def bf_plan_set_tiles(plan: int, tile_t: int = 0, group_tiles: int = 0, x_stages: int = 0):
    _check(_lib.bf_plan_set_tiles(plan, tile_t, group_tiles, x_stages))


def bf_plan_query_tiles(plan: int) -> dict:
    t, g, x, n = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(_lib.bf_plan_query_tiles(plan, ctypes.byref(t), ctypes.byref(g), ctypes.byref(x), ctypes.byref(n)))
    return {"tile_t": t.value, "group_tiles": g.value, "x_stages": x.value, "n_groups": n.value}


def bf_plan_set_weight_buffers(plan: int, n: int):
    _check(_lib.bf_plan_set_weight_buffers(plan, n))


def bf_plan_set_input_order(plan: int, perm=None):
    pa, pp = _host(perm, np.int32)
    _check(_lib.bf_plan_set_input_order(plan, pp))


def bf_plan_query(plan: int) -> dict:
    k, t, g = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    nb = ctypes.c_size_t()
    _check(_lib.bf_plan_query(plan, ctypes.byref(k), ctypes.byref(t), ctypes.byref(g), ctypes.byref(nb)))
    return {"kernel": k.value, "tile_t": t.value, "group_tiles": g.value, "device_bytes": nb.value}


def bf_export_weights(plan: int, d_w: int, d_scale: int = 0):
    _check(_lib.bf_export_weights(plan, d_w, d_scale or None))


def bf_corner_turn(d_in: int, in_dtype: int, d_out: int, out_dtype: int, n_ant: int, n_chan: int,
                   n_samp: int, perm=None, stream: int = 0):
    pa, pp = _host(perm, np.int32)
    _check(_lib.bf_corner_turn(d_in, in_dtype, d_out, out_dtype, n_ant, n_chan, n_samp, pp,
                               stream or None))


def bf_batch_create(plans, tile_t: int = 0) -> int:
    arr = (ctypes.c_void_p * len(plans))(*plans)
    b = ctypes.c_void_p()
    _check(_lib.bf_batch_create(ctypes.byref(b), arr, len(plans), tile_t))
    return b.value


def bf_batch_set(batch: int, job: int, d_voltages: int, n_samp: int, d_power: int):
    _check(_lib.bf_batch_set(batch, job, d_voltages or None, n_samp, d_power or None))


def bf_batch_execute(batch: int, stream: int = 0):
    _check(_lib.bf_batch_execute(batch, stream or None))


def bf_batch_capture(batch: int, stream: int):
    _check(_lib.bf_batch_capture(batch, stream or None))


def bf_batch_replay(batch: int, stream: int = 0):
    _check(_lib.bf_batch_replay(batch, stream or None))


def bf_batch_sync(batch: int):
    _check(_lib.bf_batch_sync(batch))


def bf_batch_query(batch: int) -> dict:
    t, u, f = ctypes.c_int(), ctypes.c_longlong(), ctypes.c_double()
    _check(_lib.bf_batch_query(batch, ctypes.byref(t), ctypes.byref(u), ctypes.byref(f)))
    return {"tile_t": t.value, "units": u.value, "flops": f.value}


def bf_batch_destroy(batch: int):
    _check(_lib.bf_batch_destroy(batch))


def bf_server_create(plans, mem_bytes: int, max_steps: int = 3, tile_t: int = 0) -> int:
    arr = (ctypes.c_void_p * len(plans))(*plans)
    h = ctypes.c_void_p()
    _check(_lib.bf_server_create(ctypes.byref(h), arr, len(plans), mem_bytes, max_steps, tile_t))
    return h.value


def bf_server_submit(server: int, config: int, h_voltages: int, n_samp: int, h_power: int) -> int:
    i = ctypes.c_longlong()
    _check(_lib.bf_server_submit(server, config, h_voltages, n_samp, h_power, ctypes.byref(i)))
    return i.value


_COMPLETION_FIELDS = [f for f, _ in bf_completion._fields_]


def bf_server_poll(server: int, max_n: int = 256, timeout_ms: int = 0) -> list:
    buf = (bf_completion * max_n)()
    n = ctypes.c_int()
    _check(_lib.bf_server_poll(server, buf, max_n, ctypes.byref(n), timeout_ms))
    return [{f: getattr(buf[i], f) for f in _COMPLETION_FIELDS} for i in range(n.value)]


def bf_server_pause(server: int, paused: bool = True):
    _check(_lib.bf_server_pause(server, int(bool(paused))))


def bf_server_drain(server: int, timeout_ms: int = 60000):
    _check(_lib.bf_server_drain(server, timeout_ms))


def bf_server_stats(server: int) -> dict:
    c = bf_server_counters()
    _check(_lib.bf_server_stats(server, ctypes.byref(c)))
    return {f: getattr(c, f) for f, _ in bf_server_counters._fields_}


def bf_server_destroy(server: int):
    _check(_lib.bf_server_destroy(server))


def bf_server_now() -> float:
    return _lib.bf_server_now()


def bf_detect(d_power: int, n_beam: int, n_chan: int, n_win: int, k_sigma: float, d_z: int, d_hits: int,
              max_hits: int, d_n_hits: int, stream: int = 0):
    _check(_lib.bf_detect(d_power or None, n_beam, n_chan, n_win, float(k_sigma), d_z or None, d_hits or None,
                          max_hits, d_n_hits or None, stream or None))


def detect(power, k_sigma: float, max_hits: int = 1 << 16, want_z: bool = True, stream=None):
    """Torch helper around bf_detect: power is a device float32 tensor
    [B][C][T_o]; returns (z or None, hits [n][3] int32 tensor, total hit count)."""
    import torch
    B, C, W = power.shape
    s = stream if stream is not None else torch.cuda.current_stream()
    z = torch.empty_like(power) if want_z else None
    hits = torch.empty((max_hits, 3), dtype=torch.int32, device=power.device)
    n = torch.zeros(1, dtype=torch.int32, device=power.device)
    bf_detect(power.data_ptr(), B, C, W, k_sigma, z.data_ptr() if want_z else 0, hits.data_ptr(), max_hits,
              n.data_ptr(), s.cuda_stream)
    total = int(n.item())
    return z, hits[:min(total, max_hits)], total


def bf_selftest_timeout(limit_ms: float = 50.0, stream: int = 0):
    _check(_lib.bf_selftest_timeout(float(limit_ms), stream or None))


def bf_measure_ffma(seconds: float = 1.0, stream: int = 0) -> float:
    """The GPU's FP32 FFMA rate in TFLOP/s (a measurement aid)."""
    v = ctypes.c_double(0.0)
    _check(_lib.bf_measure_ffma(float(seconds), ctypes.byref(v), stream or None))
    return v.value


# ------------------------------------------------------------ torch helper
class Plan:
    """A beamforming plan on the current CUDA device.  Voltages are torch
    tensors whose bytes hold the plan's dtype (for example float16 [C][T][2N]
    for BF_C16F, int8 [C][T][2N] for BF_CI8, uint8 [C][T][N] for BF_CI4)."""

    def __init__(self, pos_m, freqs_hz, dirs, dtype: int, t_int: int, layout: int = BF_LAYOUT_CTN,
                 mask=None, stream=None):
        import torch
        self._torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.N = int(np.asarray(pos_m).shape[0])
        self.C = int(np.asarray(freqs_hz).shape[0])
        self.B = int(np.asarray(dirs).shape[0])
        self.dtype, self.t_int, self.layout = dtype, t_int, layout
        self.handle = bf_plan_create(pos_m, freqs_hz, dirs, dtype, t_int, layout, mask,
                                     self.stream.cuda_stream)

    def close(self):
        if self.handle:
            bf_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def n_samp(self, x) -> int:
        per = SAMPLE_BYTES[self.dtype] * self.N * self.C
        nbytes = x.numel() * x.element_size()
        if nbytes % per:
            raise ValueError("voltage tensor size does not match the plan")
        return nbytes // per

    def execute(self, x, out=None, n_samp=None):
        T = self.n_samp(x) if n_samp is None else n_samp
        if out is None:
            out = self._torch.empty((self.B, self.C, T // self.t_int), dtype=self._torch.float32,
                                    device=x.device)
        bf_execute(self.handle, x.data_ptr(), T, out.data_ptr(), self.stream.cuda_stream)
        return out

    def execute_complex(self, x, out=None, n_samp=None):
        T = self.n_samp(x) if n_samp is None else n_samp
        if out is None:
            out = self._torch.empty((self.B, self.C, T, 2), dtype=self._torch.float32, device=x.device)
        bf_execute_complex(self.handle, x.data_ptr(), T, out.data_ptr(), self.stream.cuda_stream)
        return out

    def execute_incoherent(self, x, out=None, n_samp=None):
        T = self.n_samp(x) if n_samp is None else n_samp
        if out is None:
            out = self._torch.empty((self.C, T // self.t_int), dtype=self._torch.float32, device=x.device)
        bf_execute_incoherent(self.handle, x.data_ptr(), T, out.data_ptr(), self.stream.cuda_stream)
        return out

    def execute_host(self, x_host, out_host=None, n_samp=None):
        """x_host: numpy array or pinned CPU tensor; returns the host powers."""
        torch = self._torch
        if isinstance(x_host, np.ndarray):
            x_host = torch.from_numpy(np.ascontiguousarray(x_host))
        T = self.n_samp(x_host) if n_samp is None else n_samp
        if out_host is None:
            out_host = torch.empty((self.B, self.C, T // self.t_int), dtype=torch.float32)
        bf_execute_host(self.handle, x_host.data_ptr(), T, out_host.data_ptr())
        return out_host

    def weights(self, dirs=None):
        bf_weights(self.handle, dirs)

    def set_kernel(self, kernel: int, tile_t: int = 0):
        bf_plan_set_kernel(self.handle, kernel, tile_t)

    def set_tiles(self, tile_t: int = 0, group_tiles: int = 0, x_stages: int = 0):
        bf_plan_set_tiles(self.handle, tile_t, group_tiles, x_stages)

    def query_tiles(self) -> dict:
        return bf_plan_query_tiles(self.handle)

    def set_weight_buffers(self, n: int):
        bf_plan_set_weight_buffers(self.handle, n)

    def set_input_order(self, perm):
        bf_plan_set_input_order(self.handle, perm)

    def query(self) -> dict:
        return bf_plan_query(self.handle)

    def export_weights(self):
        torch = self._torch
        w = torch.empty((self.C, self.B, self.N, 2), dtype=torch.float32, device="cuda")
        s = torch.empty((self.C, self.B), dtype=torch.float32, device="cuda")
        bf_export_weights(self.handle, w.data_ptr(), s.data_ptr())
        return w, s

    def sync(self):
        bf_sync(self.handle)


class Batch:
    """Several plans stepped together (``bf_batch_*``): one call, or one
    CUDA graph replay, per step, scheduled by job size.
    ``set(j, x, out)`` binds job j's voltages and powers (torch tensors);
    ``execute()`` runs one step on the stream given here; ``capture()`` /
    ``replay()`` record and relaunch that step as a CUDA graph."""

    def __init__(self, plans, tile_t: int = 0, stream=None):
        import torch
        self._torch = torch
        self.plans = list(plans)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.handle = bf_batch_create([p.handle for p in self.plans], tile_t)
        self._bound = [None] * len(self.plans)

    def set(self, job: int, x, out=None, n_samp=None):
        p = self.plans[job]
        T = p.n_samp(x) if n_samp is None else n_samp
        if out is None:
            out = self._torch.empty((p.B, p.C, T // p.t_int), dtype=self._torch.float32, device=x.device)
        bf_batch_set(self.handle, job, x.data_ptr(), T, out.data_ptr())
        self._bound[job] = (x, out)   # keeps the bound tensors alive
        return out

    def execute(self):
        bf_batch_execute(self.handle, self.stream.cuda_stream)

    def capture(self):
        bf_batch_capture(self.handle, self.stream.cuda_stream)

    def replay(self):
        bf_batch_replay(self.handle, self.stream.cuda_stream)

    def sync(self):
        bf_batch_sync(self.handle)

    def query(self) -> dict:
        return bf_batch_query(self.handle)

    def close(self):
        if self.handle:
            bf_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Serving loop over several plans (``bf_server_*``).  ``submit`` takes a
    host tensor of one chunk (page-locked for asynchronous copies) and a host
    float32 tensor with room for [B][C][ceil(T / T_int)] powers; both must
    stay alive until the chunk's completion has been polled."""

    def __init__(self, plans, mem_bytes: int, max_steps: int = 3, tile_t: int = 0):
        self.plans = list(plans)
        self.handle = bf_server_create([p.handle for p in self.plans], int(mem_bytes), max_steps, tile_t)
        self._live = {}

    def submit(self, config: int, x_host, out_host, n_samp=None) -> int:
        p = self.plans[config]
        T = p.n_samp(x_host) if n_samp is None else n_samp
        i = bf_server_submit(self.handle, config, x_host.data_ptr(), T, out_host.data_ptr())
        self._live[i] = (x_host, out_host)
        return i

    def poll(self, max_n: int = 256, timeout_ms: int = 0) -> list:
        done = bf_server_poll(self.handle, max_n, timeout_ms)
        for c in done:
            self._live.pop(c["id"], None)
        return done

    def drain(self, timeout_ms: int = 60000):
        bf_server_drain(self.handle, timeout_ms)

    def pause(self, paused: bool = True):
        bf_server_pause(self.handle, paused)

    def stats(self) -> dict:
        return bf_server_stats(self.handle)

    def close(self):
        if self.handle:
            bf_server_destroy(self.handle)
            self.handle = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
