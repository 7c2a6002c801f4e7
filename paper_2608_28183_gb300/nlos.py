"""Thin Python binding of the C ABI in include/nlos.h (argument marshalling only).

Every step of a reconstruction runs in the CUDA library's kernels; this module
only checks tensors, passes raw pointers and the current CUDA stream, and turns
status codes into exceptions. If the library is missing it raises: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnlos_gb300.so")

NLOS_FK, NLOS_PHASOR_RSD, NLOS_PHASOR_DENSE = 0, 1, 2
NLOS_F32, NLOS_F16, NLOS_BF16 = 0, 1, 2
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OUT_OF_MEMORY", 3: "CUDA", 4: "UNSUPPORTED", 5: "TIMEOUT"}
METHODS = {"fk": NLOS_FK, "pf": NLOS_PHASOR_RSD, "phasor": NLOS_PHASOR_RSD, "pf_dense": NLOS_PHASOR_DENSE}
STORAGES = {"f32": NLOS_F32, "f16": NLOS_F16, "bf16": NLOS_BF16}
OUTPUTS = {"magnitude": 0, "complex": 1}
PLAN_NO_WORKSPACE, PLAN_SEPARATE_AXES = 1, 2
# bounds-checked debug build (NLOS_BOUNDS_CHECK=1): plans read their device
# error word when closed and record nonzero codes here
BOUNDS_CHECKED = os.environ.get("NLOS_BOUNDS_CHECK", "0") not in ("", "0")
WORKSPACE_ERRORS = []

EXPORTED = ["nlos_plan_desc_default", "nlos_plan_create", "nlos_plan_query", "nlos_reconstruct",
            "nlos_reconstruct_ws", "nlos_reconstruct_host", "nlos_reconstruct_batch",
            "nlos_plan_set_profiling", "nlos_plan_stage_times", "nlos_plan_stage_name",
            "nlos_plan_destroy", "nlos_last_error", "nlos_version", "nlos_reconstruct_noalloc",
            "nlos_plan_autotune", "nlos_plan_get_tiles", "nlos_plan_set_tiles",
            "nlos_batch_create", "nlos_batch_launch", "nlos_batch_destroy", "nlos_plan_create_ex",
            "nlos_server_create", "nlos_server_preload", "nlos_server_submit", "nlos_server_wait",
            "nlos_server_stats", "nlos_server_destroy", "nlos_workspace_check", "nlos_selftest_bounded_wait",
            "nlos_max_image", "nlos_moe_mix", "nlos_coherence_merge", "nlos_dda",
            "nlos_bin_transient", "nlos_bin_phasors", "nlos_plan_band", "nlos_reconstruct_phasors",
            "nlos_reconstruct_host_many", "nlos_debug_fail_allocation", "nlos_selftest_umma",
            "nlos_ffma_rate_launch", "nlos_plan_memory", "nlos_server_memory", "nlos_selftest_bounds",
            "nlos_reconstruct_moe"]


class PlanDesc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nt", ctypes.c_int),
        ("bin_width_s", ctypes.c_double),
        ("wall_w_m", ctypes.c_double), ("wall_h_m", ctypes.c_double),
        ("method", ctypes.c_int), ("storage", ctypes.c_int), ("pad_factor", ctypes.c_int),
        ("wavelength_m", ctypes.c_double), ("cycles", ctypes.c_double),
        ("n_depths", ctypes.c_int),
        ("depth_min_m", ctypes.c_double), ("depth_max_m", ctypes.c_double),
        ("sigma_s", ctypes.c_int), ("sigma_t", ctypes.c_int),
        ("delta_m", ctypes.c_double),
        ("output", ctypes.c_int),
    ]


class NlosError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libnlos_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run paper_2608_28183_gb300/build.py)")
    lib = ctypes.CDLL(path)
    vp, sz = ctypes.c_void_p, ctypes.c_size_t
    lib.nlos_plan_desc_default.argtypes = [ctypes.POINTER(PlanDesc)]
    lib.nlos_plan_desc_default.restype = None
    lib.nlos_plan_create.argtypes = [ctypes.POINTER(PlanDesc), ctypes.POINTER(vp)]
    lib.nlos_plan_query.argtypes = [vp, ctypes.POINTER(sz * 3), ctypes.POINTER(sz), ctypes.POINTER(sz),
                                    ctypes.POINTER(sz)]
    lib.nlos_reconstruct.argtypes = [vp, vp, vp, vp]
    lib.nlos_reconstruct_ws.argtypes = [vp, vp, vp, vp, sz, vp]
    lib.nlos_reconstruct_host.argtypes = [vp, vp, vp, vp]
    lib.nlos_reconstruct_batch.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                           ctypes.POINTER(vp), ctypes.c_int, vp]
    lib.nlos_plan_destroy.argtypes = [vp]
    lib.nlos_reconstruct_noalloc.argtypes = [vp, vp, vp, vp]
    lib.nlos_reconstruct_noalloc.restype = ctypes.c_int
    lib.nlos_plan_autotune.argtypes = [vp, vp]
    lib.nlos_plan_get_tiles.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    lib.nlos_plan_set_tiles.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.c_int]
    lib.nlos_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.c_int,
                                      ctypes.c_int, ctypes.POINTER(vp)]
    lib.nlos_batch_launch.argtypes = [vp, vp]
    lib.nlos_batch_destroy.argtypes = [vp]
    lib.nlos_plan_create_ex.argtypes = [ctypes.POINTER(PlanDesc), ctypes.c_int, ctypes.POINTER(vp)]
    lib.nlos_server_create.argtypes = [sz, ctypes.c_int, ctypes.POINTER(vp)]
    lib.nlos_server_preload.argtypes = [vp, ctypes.POINTER(PlanDesc)]
    lib.nlos_server_submit.argtypes = [vp, ctypes.POINTER(PlanDesc), vp, vp, ctypes.POINTER(ctypes.c_uint64)]
    lib.nlos_server_wait.argtypes = [vp, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    lib.nlos_server_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_ulonglong), ctypes.c_int]
    lib.nlos_server_destroy.argtypes = [vp]
    lib.nlos_workspace_check.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int)]
    lib.nlos_workspace_check.restype = ctypes.c_int
    lib.nlos_selftest_bounded_wait.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    lib.nlos_selftest_bounded_wait.restype = ctypes.c_int
    ll, fl = ctypes.c_longlong, ctypes.c_float
    lib.nlos_max_image.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp]
    lib.nlos_moe_mix.argtypes = [vp, vp, ll, fl, fl, vp, vp]
    lib.nlos_coherence_merge.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ll, fl, vp, vp, vp]
    lib.nlos_dda.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ll, ctypes.c_int, vp, vp]
    u32 = ctypes.c_uint32
    lib.nlos_bin_transient.argtypes = [vp, vp, ll, ctypes.c_int, ctypes.c_int, ctypes.c_int, u32, u32, ctypes.c_int,
                                       vp, vp]
    lib.nlos_bin_phasors.argtypes = [vp, vp, vp, ll, u32, u32, ctypes.c_int, vp, vp]
    lib.nlos_plan_band.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.nlos_reconstruct_phasors.argtypes = [vp, vp, vp, vp]
    lib.nlos_reconstruct_moe.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    lib.nlos_reconstruct_host_many.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.c_int, vp]
    lib.nlos_debug_fail_allocation.argtypes = [ctypes.c_int]
    lib.nlos_debug_fail_allocation.restype = None
    lib.nlos_selftest_umma.argtypes = [ctypes.c_int, vp, ctypes.POINTER(ctypes.c_int)]
    lib.nlos_selftest_umma.restype = ctypes.c_int
    lib.nlos_ffma_rate_launch.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double), vp]
    lib.nlos_ffma_rate_launch.restype = ctypes.c_int
    for name in ("nlos_max_image", "nlos_moe_mix", "nlos_coherence_merge", "nlos_dda", "nlos_bin_transient",
                 "nlos_bin_phasors", "nlos_plan_band", "nlos_reconstruct_phasors", "nlos_reconstruct_host_many",
                 "nlos_reconstruct_moe"):
        getattr(lib, name).restype = ctypes.c_int
    for name in ("nlos_plan_autotune", "nlos_plan_get_tiles", "nlos_plan_set_tiles", "nlos_batch_create",
                 "nlos_batch_launch", "nlos_batch_destroy", "nlos_plan_create_ex", "nlos_server_create",
                 "nlos_server_preload", "nlos_server_submit", "nlos_server_wait", "nlos_server_stats",
                 "nlos_server_destroy"):
        getattr(lib, name).restype = ctypes.c_int
    lib.nlos_selftest_bounds.argtypes = [ctypes.POINTER(ctypes.c_int)]
    lib.nlos_selftest_bounds.restype = ctypes.c_int
    lib.nlos_plan_memory.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    lib.nlos_plan_memory.restype = ctypes.c_int
    lib.nlos_server_memory.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t),
                                       ctypes.POINTER(ctypes.c_ulonglong)]
    lib.nlos_server_memory.restype = ctypes.c_int
    lib.nlos_plan_set_profiling.argtypes = [vp, ctypes.c_int]
    lib.nlos_plan_stage_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_longlong)]
    lib.nlos_plan_stage_name.argtypes = [vp, ctypes.c_int]
    lib.nlos_plan_stage_name.restype = ctypes.c_char_p
    for name in ("nlos_plan_create", "nlos_plan_query", "nlos_reconstruct", "nlos_reconstruct_ws",
                 "nlos_reconstruct_host", "nlos_reconstruct_batch", "nlos_plan_destroy",
                 "nlos_plan_set_profiling", "nlos_plan_stage_times"):
        getattr(lib, name).restype = ctypes.c_int
    lib.nlos_last_error.argtypes = []
    lib.nlos_last_error.restype = ctypes.c_char_p
    lib.nlos_version.argtypes = []
    lib.nlos_version.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(status: int):
    if status != 0:
        raise NlosError(status, _lib.nlos_last_error().decode())


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


@dataclass
class Geometry:
    nx: int
    ny: int
    nt: int
    bin_width_s: float
    wall_w_m: float
    wall_h_m: float


def make_desc(nx: int, ny: int, nt: int, bin_width_s: float, wall_w_m: float, wall_h_m: float,
              method: str = "fk", storage: str = "f32", pad_factor: int = 2, *,
              n_depths: int = 0, depth_min_m: float = 0.0, depth_max_m: float = 0.0,
              wavelength_m: float = 0.0, cycles: float = 5.0, sigma_s: int = 0, sigma_t: int = 0,
              delta_m: float = 0.0, output: str = "magnitude") -> PlanDesc:
    lib = load_library()
    d = PlanDesc()
    lib.nlos_plan_desc_default(ctypes.byref(d))
    d.nx, d.ny, d.nt = nx, ny, nt
    d.bin_width_s, d.wall_w_m, d.wall_h_m = bin_width_s, wall_w_m, wall_h_m
    d.method = METHODS[method]
    d.storage = STORAGES[storage]
    d.pad_factor = pad_factor
    d.wavelength_m, d.cycles = wavelength_m, cycles
    d.n_depths, d.depth_min_m, d.depth_max_m = n_depths, depth_min_m, depth_max_m
    d.sigma_s, d.sigma_t, d.delta_m = sigma_s, sigma_t, delta_m
    d.output = OUTPUTS[output]
    return d


class Plan:
    """A reconstruction plan (owns device tables and a default workspace)."""

    def __init__(self, nx: int, ny: int, nt: int, bin_width_s: float, wall_w_m: float, wall_h_m: float,
                 method: str = "fk", storage: str = "f32", pad_factor: int = 2, separate_axes: bool = False,
                 **kw):
        lib = load_library()
        d = make_desc(nx, ny, nt, bin_width_s, wall_w_m, wall_h_m, method, storage, pad_factor, **kw)
        self.desc = d
        self.method = method
        self.storage = storage
        h = ctypes.c_void_p()
        flags = PLAN_SEPARATE_AXES if separate_axes else 0
        self._own_ws = True
        _check(lib.nlos_plan_create_ex(ctypes.byref(d), flags, ctypes.byref(h)))
        self._h = h
        shape = (ctypes.c_size_t * 3)()
        ws, ib, ob = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
        _check(lib.nlos_plan_query(h, ctypes.byref(shape), ctypes.byref(ws), ctypes.byref(ib), ctypes.byref(ob)))
        self.out_shape = tuple(int(v) for v in shape)
        self.workspace_bytes = ws.value
        self.input_bytes = ib.value
        self.output_bytes = ob.value

    @property
    def handle(self):
        return self._h

    @property
    def resident_bytes(self) -> int:
        """Device memory the plan holds (tables, kernels, workspace)."""
        v = ctypes.c_size_t()
        _check(_lib.nlos_plan_memory(self._h, ctypes.byref(v)))
        return v.value

    def input_dtype(self):
        import torch
        return {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[self.storage]

    def output_dtype(self):
        import torch
        return torch.complex64 if self.desc.output == OUTPUTS["complex"] else torch.float32

    def _check_io(self, transient, volume):
        d = self.desc
        if not (transient.is_cuda and volume.is_cuda):
            raise ValueError("transient and volume must be CUDA tensors")
        if transient.dtype != self.input_dtype() or not transient.is_contiguous() \
                or tuple(transient.shape) != (d.nx, d.ny, d.nt):
            raise ValueError(f"transient must be contiguous {self.input_dtype()} [{d.nx},{d.ny},{d.nt}]")
        if volume.dtype != self.output_dtype() or not volume.is_contiguous() or tuple(volume.shape) != self.out_shape:
            raise ValueError(f"volume must be contiguous {self.output_dtype()} {list(self.out_shape)}")

    def empty_volume(self):
        import torch
        return torch.empty(self.out_shape, dtype=self.output_dtype(), device="cuda")

    def reconstruct(self, transient, volume=None, stream=None, workspace=None):
        """Reconstruct on the device; returns the volume tensor (asynchronous)."""
        if volume is None:
            volume = self.empty_volume()
        self._check_io(transient, volume)
        if workspace is None:
            _check(_lib.nlos_reconstruct(self._h, ctypes.c_void_p(transient.data_ptr()),
                                         ctypes.c_void_p(volume.data_ptr()), _stream_ptr(stream)))
        else:
            _check(_lib.nlos_reconstruct_ws(self._h, ctypes.c_void_p(transient.data_ptr()),
                                            ctypes.c_void_p(volume.data_ptr()),
                                            ctypes.c_void_p(workspace.data_ptr()),
                                            ctypes.c_size_t(workspace.numel() * workspace.element_size()),
                                            _stream_ptr(stream)))
        return volume

    def reconstruct_host(self, transient_host, volume_host, stream=None):
        """End-to-end call on host buffers (numpy arrays or CPU tensors); synchronous."""
        def ptr(x):
            return ctypes.c_void_p(x.data_ptr() if hasattr(x, "data_ptr") else x.ctypes.data)
        _check(_lib.nlos_reconstruct_host(self._h, ptr(transient_host), ptr(volume_host), _stream_ptr(stream)))
        return volume_host

    @property
    def band(self):
        """(k_lo, F): first DFT bin and number of band frequencies (phasor-field plans)."""
        k, f = ctypes.c_int(), ctypes.c_int()
        _check(_lib.nlos_plan_band(self._h, ctypes.byref(k), ctypes.byref(f)))
        return k.value, f.value

    def empty_phasors(self):
        import torch
        d = self.desc
        return torch.empty((d.nx, d.ny, self.band[1]), dtype=torch.complex64, device="cuda")

    def bin_phasors(self, pixel, ticks, t0_ticks: int, ticks_per_bin: int, phasors=None, accumulate=False,
                    route: str = "auto", stream=None):
        """Photon records into the compact phasor field [nx, ny, F]; route is
        "auto", "direct" (per photon) or "histogram" (atomic histogram + FFT)."""
        _check_photons(pixel, ticks)
        if phasors is None:
            phasors = self.empty_phasors()
        d = self.desc
        if phasors.dtype != _torch().complex64 or not phasors.is_contiguous() \
                or tuple(phasors.shape) != (d.nx, d.ny, self.band[1]):
            raise ValueError("phasors must be contiguous complex64 [nx, ny, F]")
        _check(_lib.nlos_bin_phasors(self._h, ctypes.c_void_p(pixel.data_ptr()), ctypes.c_void_p(ticks.data_ptr()),
                                     pixel.numel(), t0_ticks, ticks_per_bin,
                                     int(bool(accumulate)) | {"auto": 0, "direct": 2, "histogram": 4}[route],
                                     ctypes.c_void_p(phasors.data_ptr()), _stream_ptr(stream)))
        return phasors

    def reconstruct_phasors(self, phasors, volume=None, stream=None):
        """Reconstruct from a compact phasor field (the band transform is skipped)."""
        if volume is None:
            volume = self.empty_volume()
        if volume.dtype != self.output_dtype() or not volume.is_contiguous() or tuple(volume.shape) != self.out_shape:
            raise ValueError(f"volume must be contiguous {self.output_dtype()} {list(self.out_shape)}")
        _check(_lib.nlos_reconstruct_phasors(self._h, ctypes.c_void_p(phasors.data_ptr()),
                                             ctypes.c_void_p(volume.data_ptr()), _stream_ptr(stream)))
        return volume

    def reconstruct_host_many(self, transients_host, volumes_host, stream=None):
        """Pipelined end-to-end calls on lists of host buffers (page-locked for
        overlap); synchronous. Copies in, reconstructions and copies out of
        consecutive captures overlap."""
        if len(transients_host) != len(volumes_host):
            raise ValueError("one output buffer per input")

        def ptr(x):
            return x.data_ptr() if hasattr(x, "data_ptr") else x.ctypes.data
        for t, v in zip(transients_host, volumes_host):
            nb_t = t.numel() * t.element_size() if hasattr(t, "numel") else t.nbytes
            nb_v = v.numel() * v.element_size() if hasattr(v, "numel") else v.nbytes
            if nb_t != self.input_bytes or nb_v != self.output_bytes:
                raise ValueError(f"host buffers must hold {self.input_bytes} / {self.output_bytes} bytes")
        n = len(transients_host)
        T = (ctypes.c_void_p * n)(*[ptr(t) for t in transients_host])
        V = (ctypes.c_void_p * n)(*[ptr(v) for v in volumes_host])
        _check(_lib.nlos_reconstruct_host_many(self._h, T, V, n, _stream_ptr(stream)))
        return volumes_host

    def set_profiling(self, enable: bool):
        """Record a CUDA event after every stage of each reconstruction."""
        _check(_lib.nlos_plan_set_profiling(self._h, int(bool(enable))))

    def stage_times(self):
        """{stage name: accumulated ms} over the profiled calls, and the call count (resets)."""
        cap = 16
        times = (ctypes.c_double * cap)()
        ns, calls = ctypes.c_int(), ctypes.c_longlong()
        _check(_lib.nlos_plan_stage_times(self._h, times, cap, ctypes.byref(ns), ctypes.byref(calls)))
        names = [_lib.nlos_plan_stage_name(self._h, i).decode() for i in range(ns.value)]
        return {nm: times[i] for i, nm in enumerate(names)}, calls.value

    def autotune(self, stream=None):
        """Pick each stage's fastest launch shape (cached per plan shape)."""
        _check(_lib.nlos_plan_autotune(self._h, _stream_ptr(stream)))
        return self.tiles

    @property
    def tiles(self):
        buf = (ctypes.c_int * 16)()
        n = ctypes.c_int()
        _check(_lib.nlos_plan_get_tiles(self._h, buf, 16, ctypes.byref(n)))
        return [buf[i] for i in range(n.value)]

    @tiles.setter
    def tiles(self, values):
        arr = (ctypes.c_int * len(values))(*values)
        _check(_lib.nlos_plan_set_tiles(self._h, arr, len(values)))

    def check_workspace(self) -> int:
        """Read and clear the default workspace's device error word (0: clean;
        1, 2: a bounded wait ran out; 3: bounds-checked build, an index fell
        outside its buffer)."""
        code = ctypes.c_int(0)
        _lib.nlos_workspace_check(self._h, None, ctypes.byref(code))
        return code.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            if BOUNDS_CHECKED and self.workspace_bytes and self._own_ws:
                code = self.check_workspace()
                if code:
                    WORKSPACE_ERRORS.append((self.method, self.desc.nx, self.desc.ny, self.desc.nt, code))
            _check(_lib.nlos_plan_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def reconstruct_batch(plans, transients, volumes, workspaces=None, stream=None):
    """Reconstruct several captures forked over the library's streams (asynchronous)."""
    n = len(plans)
    P = (ctypes.c_void_p * n)(*[p.handle.value for p in plans])
    T = (ctypes.c_void_p * n)(*[t.data_ptr() for t in transients])
    V = (ctypes.c_void_p * n)(*[v.data_ptr() for v in volumes])
    for p, t, v in zip(plans, transients, volumes):
        p._check_io(t, v)
    W = None if workspaces is None else (ctypes.c_void_p * n)(*[w.data_ptr() for w in workspaces])
    _check(_lib.nlos_reconstruct_batch(P, T, V, W, n, _stream_ptr(stream)))
    return volumes


class Batch:
    """Many reconstructions recorded once into a CUDA graph and replayed.

    The device buffers given here are the batch's inputs and outputs for its
    whole life; launch() replays the graph on the current stream."""

    def __init__(self, plans, transients, volumes, max_streams: int = 0):
        load_library()
        n = len(plans)
        for p, t, v in zip(plans, transients, volumes):
            p._check_io(t, v)
        self._keep = (list(plans), list(transients), list(volumes))
        P = (ctypes.c_void_p * n)(*[p.handle.value for p in plans])
        T = (ctypes.c_void_p * n)(*[t.data_ptr() for t in transients])
        V = (ctypes.c_void_p * n)(*[v.data_ptr() for v in volumes])
        h = ctypes.c_void_p()
        _check(_lib.nlos_batch_create(P, T, V, n, max_streams, ctypes.byref(h)))
        self._h = h

    def launch(self, stream=None):
        _check(_lib.nlos_batch_launch(self._h, _stream_ptr(stream)))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _check(_lib.nlos_batch_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server: queue requests from any thread, wait for tickets."""

    def __init__(self, memory_budget_bytes: int, n_slots: int = 8):
        load_library()
        h = ctypes.c_void_p()
        _check(_lib.nlos_server_create(ctypes.c_size_t(memory_budget_bytes), n_slots, ctypes.byref(h)))
        self._h = h

    def preload(self, desc: PlanDesc):
        _check(_lib.nlos_server_preload(self._h, ctypes.byref(desc)))

    def submit(self, desc: PlanDesc, transient, volume) -> int:
        t = ctypes.c_uint64()
        _check(_lib.nlos_server_submit(self._h, ctypes.byref(desc), ctypes.c_void_p(transient.data_ptr()),
                                       ctypes.c_void_p(volume.data_ptr()), ctypes.byref(t)))
        return t.value

    def wait(self, ticket: int, timeout_s: float = 60.0) -> float:
        lat = ctypes.c_double()
        _check(_lib.nlos_server_wait(self._h, ctypes.c_uint64(ticket), timeout_s, ctypes.byref(lat)))
        return lat.value

    def memory(self) -> dict:
        pb, wb, ev = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_ulonglong()
        _check(_lib.nlos_server_memory(self._h, ctypes.byref(pb), ctypes.byref(wb), ctypes.byref(ev)))
        return {"plan_bytes": pb.value, "workspace_bytes": wb.value, "evictions": ev.value}

    def stats(self, reset: bool = False) -> dict:
        p50, p99, vps = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        n = ctypes.c_ulonglong()
        _check(_lib.nlos_server_stats(self._h, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(vps),
                                      ctypes.byref(n), int(reset)))
        return {"p50_ms": p50.value, "p99_ms": p99.value, "volumes_per_s": vps.value, "completed": n.value}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _check(_lib.nlos_server_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def desc_for_capture(geom, method="fk", storage="f32", **kw) -> PlanDesc:
    return make_desc(geom.nx, geom.ny, geom.nt, geom.bin_width_s, geom.wall_w_m, geom.wall_h_m,
                     method=method, storage=storage, **kw)


def plan_for_capture(geom, method="fk", storage="f32", **kw) -> Plan:
    return Plan(geom.nx, geom.ny, geom.nt, geom.bin_width_s, geom.wall_w_m, geom.wall_h_m,
                method=method, storage=storage, **kw)


def version() -> str:
    return load_library().nlos_version().decode()


# ---------------------------------------------------------------------------
# Post-processing (Sec. 4.4 and the display reduction of Sec. 4.2)
# ---------------------------------------------------------------------------

def _dev_f32(x, name, dtype=None):
    import torch
    dt = torch.float32 if dtype is None else dtype
    if not x.is_cuda or x.dtype != dt or not x.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA {dt} tensor")


def max_image(volume, take_sqrt: bool = False, image=None, stream=None):
    """f(x, y) = max_z v(x, y, z) of a float32 [nx, ny, nz] volume (sqrt of it if take_sqrt)."""
    import torch
    load_library()
    _dev_f32(volume, "volume")
    nx, ny, nz = volume.shape
    if image is None:
        image = torch.empty((nx, ny), dtype=torch.float32, device=volume.device)
    _dev_f32(image, "image")
    if tuple(image.shape) != (nx, ny):
        raise ValueError("image must be [nx, ny]")
    _check(_lib.nlos_max_image(ctypes.c_void_p(volume.data_ptr()), nx, ny, nz, int(bool(take_sqrt)),
                               ctypes.c_void_p(image.data_ptr()), _stream_ptr(stream)))
    return image


def reconstruct_moe(fk_plan, pf_plan, transient, volume_fk=None, volume_pf=None, stream=None, stream2=None):
    """Both experts of the mixture (Sec. 4.4) from one transient with the
    lateral forward transform shared: f-k on `stream`, the phasor branch on
    `stream2` (None: after the f-k branch on `stream`); `stream` waits for
    both. Float32 plans with their own workspaces, same grid and padding.
    Returns (volume_fk, volume_pf)."""
    if volume_fk is None:
        volume_fk = fk_plan.empty_volume()
    if volume_pf is None:
        volume_pf = pf_plan.empty_volume()
    fk_plan._check_io(transient, volume_fk)
    pf_plan._check_io(transient, volume_pf)
    s1 = _stream_ptr(stream)
    s2 = s1 if stream2 is None else _stream_ptr(stream2)
    _check(_lib.nlos_reconstruct_moe(fk_plan._h, pf_plan._h, ctypes.c_void_p(transient.data_ptr()),
                                     ctypes.c_void_p(volume_fk.data_ptr()), ctypes.c_void_p(volume_pf.data_ptr()),
                                     s1, s2))
    return volume_fk, volume_pf


def moe_mix(img_fk, img_rsd, beta: float = 0.3, eps: float = 1e-3, out=None, stream=None):
    """Eq. 10 on max-normalised images; the result is normalised to peak 1."""
    import torch
    load_library()
    _dev_f32(img_fk, "img_fk")
    _dev_f32(img_rsd, "img_rsd")
    if img_fk.shape != img_rsd.shape:
        raise ValueError("images must have the same shape")
    if out is None:
        out = torch.empty_like(img_fk)
    _dev_f32(out, "out")
    _check(_lib.nlos_moe_mix(ctypes.c_void_p(img_fk.data_ptr()), ctypes.c_void_p(img_rsd.data_ptr()),
                             img_fk.numel(), beta, eps, ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def coherence_merge(frames, eps: float = 1e-6, merged=None, coherence=None, stream=None):
    """Eqs. 8-9 over N_w complex64 volumes of one shape: returns (merged, coherence)."""
    import torch
    load_library()
    for f in frames:
        _dev_f32(f, "frame", torch.complex64)
        if f.shape != frames[0].shape:
            raise ValueError("frames must have one shape")
    shape = frames[0].shape
    if merged is None:
        merged = torch.empty(shape, dtype=torch.float32, device=frames[0].device)
    if coherence is None:
        coherence = torch.empty(shape, dtype=torch.float32, device=frames[0].device)
    F = (ctypes.c_void_p * len(frames))(*[f.data_ptr() for f in frames])
    _check(_lib.nlos_coherence_merge(F, len(frames), frames[0].numel(), eps, ctypes.c_void_p(merged.data_ptr()),
                                     ctypes.c_void_p(coherence.data_ptr()), _stream_ptr(stream)))
    return merged, coherence


def dda(frames, out=None, stream=None):
    """Depth-dependent average of N_w float32 [nx, ny, nz] volumes, frames[0] the newest."""
    import torch
    load_library()
    for f in frames:
        _dev_f32(f, "frame")
        if f.shape != frames[0].shape:
            raise ValueError("frames must have one shape")
    shape = frames[0].shape
    if out is None:
        out = torch.empty(shape, dtype=torch.float32, device=frames[0].device)
    F = (ctypes.c_void_p * len(frames))(*[f.data_ptr() for f in frames])
    _check(_lib.nlos_dda(F, len(frames), frames[0].numel() // shape[-1], shape[-1],
                         ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


# ---------------------------------------------------------------------------
# Photon binning (Sec. 4.1)
# ---------------------------------------------------------------------------

def _torch():
    import torch
    return torch


def _check_photons(pixel, ticks):
    torch = _torch()
    for x, name in ((pixel, "pixel"), (ticks, "ticks")):
        if not x.is_cuda or x.dtype != torch.uint32 or not x.is_contiguous() or x.dim() != 1:
            raise ValueError(f"{name} must be a contiguous 1-D CUDA uint32 tensor")
    if pixel.numel() != ticks.numel():
        raise ValueError("pixel and ticks must have one length")


def bin_transient(pixel, ticks, nx: int, ny: int, nt: int, t0_ticks: int, ticks_per_bin: int, transient=None,
                  accumulate: bool = False, stream=None):
    """Histogram photon records into a float32 transient [nx, ny, nt] on the device."""
    torch = _torch()
    load_library()
    _check_photons(pixel, ticks)
    if transient is None:
        transient = torch.empty((nx, ny, nt), dtype=torch.float32, device=pixel.device)
    _dev_f32(transient, "transient")
    if tuple(transient.shape) != (nx, ny, nt):
        raise ValueError("transient must be [nx, ny, nt]")
    _check(_lib.nlos_bin_transient(ctypes.c_void_p(pixel.data_ptr()), ctypes.c_void_p(ticks.data_ptr()),
                                   pixel.numel(), nx, ny, nt, t0_ticks, ticks_per_bin, int(bool(accumulate)),
                                   ctypes.c_void_p(transient.data_ptr()), _stream_ptr(stream)))
    return transient


def ffma_rate(blocks: int = 152 * 8, iters: int = 2048, repeats: int = 5, stream=None) -> float:
    """Measured FP32 FMA throughput in TFLOP/s: best of `repeats` launches of
    the library's FMA-chain probe, timed with CUDA events on `stream`."""
    torch = _torch()
    load_library()
    s = stream if stream is not None else torch.cuda.current_stream()
    params = torch.tensor([0.9999, 1e-4, 1.0], dtype=torch.float32, device="cuda")
    sink = torch.empty(blocks * 256, dtype=torch.float32, device="cuda")
    flops = ctypes.c_double(0.0)
    best = 0.0
    for _ in range(repeats + 1):
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(s)
        _check(_lib.nlos_ffma_rate_launch(ctypes.c_void_p(params.data_ptr()), ctypes.c_void_p(sink.data_ptr()),
                                          blocks, iters, ctypes.byref(flops), ctypes.c_void_p(s.cuda_stream)))
        t1.record(s)
        t1.synchronize()
        best = max(best, flops.value / (t0.elapsed_time(t1) * 1e-3) / 1e12)
    return best
