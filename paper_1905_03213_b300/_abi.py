"""ctypes declarations of include/wproj.h and a torch-facing wrapper (marshalling only)."""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwproj.so")

WP_OK, WP_EINVAL, WP_ENOMEM, WP_ECUDA, WP_EOVERFLOW, WP_ESTATE = range(6)
WP_TABLE_F32, WP_TABLE_F16, WP_TABLE_BF16 = 0, 1, 2
WP_ACCUMULATE, WP_HERMITIAN_PAIRS, WP_KEEP_BINNING, WP_COMPENSATED = 1, 2, 4, 8
_TABLES = {"f32": WP_TABLE_F32, "f16": WP_TABLE_F16, "bf16": WP_TABLE_BF16}

# every function declared in include/wproj.h
SYMBOLS = ("wp_create", "wp_destroy", "wp_last_error", "wp_make_wkernels", "wp_grid", "wp_degrid",
           "wp_fft_to_image", "wp_plane_info", "wp_coords", "wp_wkernel_export", "wp_wkernel_norm",
           "wp_profile", "wp_profile_read", "wp_taper_eval_host", "wp_grid_noalloc", "wp_degrid_last", "wp_image_to_grid",
           "wp_batch_create", "wp_batch_grid", "wp_batch_fused_jobs", "wp_batch_destroy",
           "wp_baseline_order", "wp_grid_baseline", "wp_probe_fp32_fma")
PHASES = ("wkernels", "plan", "grid", "degrid", "fft", "image")


class WProjError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"wproj error {code}: {msg}")
        self.code = code


class Job(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("uvw", ctypes.c_void_p), ("freq", ctypes.c_void_p),
                ("vis", ctypes.c_void_p), ("weight", ctypes.c_void_p), ("nrow", ctypes.c_int64),
                ("nchan", ctypes.c_int32), ("flags", ctypes.c_int32), ("grid", ctypes.c_void_p),
                ("sum_w", ctypes.c_void_p), ("n_dropped", ctypes.c_void_p)]


class Params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("cell_rad", ctypes.c_double), ("n_w", ctypes.c_int32),
                ("w_max", ctypes.c_double), ("support_min", ctypes.c_int32), ("support_max", ctypes.c_int32),
                ("oversample", ctypes.c_int32), ("screen_m", ctypes.c_int32), ("table_type", ctypes.c_int32),
                ("tile_x", ctypes.c_int32), ("tile_y", ctypes.c_int32), ("device", ctypes.c_int32),
                ("units_per_cta", ctypes.c_int32)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1905_03213_b300/build.py "
                          "(or __graft_entry__.build()); there is no fallback implementation")
    L = ctypes.CDLL(LIB_PATH)
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    L.wp_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(Params)]
    L.wp_destroy.argtypes = [P]
    L.wp_destroy.restype = None
    L.wp_last_error.argtypes = [P]
    L.wp_last_error.restype = ctypes.c_char_p
    L.wp_make_wkernels.argtypes = [P, P]
    L.wp_grid.argtypes = [P, P, P, P, P, I64, I32, I32, P, P, P, P]
    L.wp_degrid.argtypes = [P, P, P, P, I64, I32, P, P]
    L.wp_degrid_last.argtypes = [P, P, P, P]
    L.wp_fft_to_image.argtypes = [P, P, P, I32, P, P]
    L.wp_image_to_grid.argtypes = [P, P, P, I32, P, P]
    L.wp_batch_create.argtypes = [ctypes.POINTER(Job), I32, ctypes.POINTER(P)]
    L.wp_batch_grid.argtypes = [P, P]
    L.wp_batch_fused_jobs.argtypes = [P]
    L.wp_batch_fused_jobs.restype = I32
    L.wp_batch_destroy.argtypes = [P]
    L.wp_batch_destroy.restype = None
    L.wp_plane_info.argtypes = [P, P, P]
    L.wp_baseline_order.argtypes = [P, P, P, I64, I32, P, P, P]
    L.wp_grid_baseline.argtypes = [P, P, P, P, P, P, P, I32, I64, I32, I32, P, P, P, P]
    L.wp_coords.argtypes = [P, P, P, I64, I32, I32, P, P]
    L.wp_wkernel_export.argtypes = [P, I32, I32, P, I64]
    L.wp_wkernel_norm.argtypes = [P, P]
    L.wp_profile.argtypes = [P, I32]
    L.wp_profile_read.argtypes = [P, P, P, P]
    L.wp_taper_eval_host.argtypes = [D, P, I64, P]
    L.wp_grid_noalloc.argtypes = [P, P, P, P, P, I64, I32, I32, P, P, P, P]
    L.wp_probe_fp32_fma.argtypes = [I32, I32, I64, I32, P, P]
    return L


lib = _load()


def taper_eval_host(c: float, x) -> np.ndarray:
    """The library's taper t(x) = psi_0(c, x) / psi_0(c, 0), evaluated on the host."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty_like(x)
    rc = lib.wp_taper_eval_host(c, x.ctypes.data, x.size, out.ctypes.data)
    if rc:
        raise WProjError(rc, "wp_taper_eval_host: invalid argument")
    return out


def probe_fp32_fma(device: int = 0, packed: bool = True, iters: int = 100_000, reps: int = 5):
    """Measured FP32 FMA throughput of the device: (TFLOP/s, ms per launch)."""
    tf, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    rc = lib.wp_probe_fp32_fma(device, 1 if packed else 0, iters, reps, ctypes.byref(tf), ctypes.byref(ms))
    if rc:
        raise WProjError(rc, "wp_probe_fp32_fma failed")
    return tf.value, ms.value


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dev_tensor(t, dtype, name, shape=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA torch tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t


class WProj:
    """One imaging geometry (a libwproj context) on one device."""

    def __init__(self, n: int, cell: float, n_w: int, w_max: float, support_min: int, support_max: int,
                 oversample: int, screen_m: int = 0, table: str = "f32", tile: tuple[int, int] = (0, 0),
                 device: int = 0, units_per_cta: int = 0):
        self.n, self.cell, self.n_w, self.w_max = n, cell, n_w, w_max
        self.support_min, self.support_max, self.oversample = support_min, support_max, oversample
        self.table = table
        self.device = device
        prm = Params(n, cell, n_w, w_max, support_min, support_max, oversample, screen_m, _TABLES[table],
                     tile[0], tile[1], device, units_per_cta)
        h = ctypes.c_void_p()
        rc = lib.wp_create(ctypes.byref(h), ctypes.byref(prm))
        if rc:
            raise WProjError(rc, lib.wp_last_error(None).decode())
        self._h = h

    # -- plumbing
    def _check(self, rc: int, what: str):
        if rc:
            raise WProjError(rc, f"{what}: {lib.wp_last_error(self._h).decode()}")

    def _stream(self, stream):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        return ctypes.c_void_p(s.cuda_stream)

    def close(self):
        if getattr(self, "_h", None):
            lib.wp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- the calls of include/wproj.h
    def make_wkernels(self, stream=None):
        self._check(lib.wp_make_wkernels(self._h, self._stream(stream)), "wp_make_wkernels")

    def grid(self, uvw, freq, vis, weight=None, grid=None, sum_w=None, n_dropped=None,
             hermitian_pairs: bool = False, accumulate: bool = False, keep_binning: bool = False,
             compensated: bool = False, stream=None):
        """Returns (grid [N, N] complex64, sum_w [1] float64, n_dropped [1] int64), device tensors.
        keep_binning: keep the binning for degrid_last (WP_KEEP_BINNING); compensated: compensated
        float32 accumulation of the grid (WP_COMPENSATED)."""
        import torch
        dev = torch.device("cuda", self.device)
        _dev_tensor(uvw, torch.float64, "uvw")
        nrow = uvw.shape[0]
        _dev_tensor(freq, torch.float64, "freq")
        nchan = freq.shape[0]
        _dev_tensor(vis, torch.complex64, "vis", (nrow, nchan))
        if weight is not None:
            _dev_tensor(weight, torch.float32, "weight", (nrow, nchan))
        if grid is None:
            grid = torch.empty((self.n, self.n), dtype=torch.complex64, device=dev)
        _dev_tensor(grid, torch.complex64, "grid", (self.n, self.n))
        if sum_w is None:
            sum_w = torch.zeros(1, dtype=torch.float64, device=dev)
        if n_dropped is None:
            n_dropped = torch.zeros(1, dtype=torch.int64, device=dev)
        flags = ((WP_ACCUMULATE if accumulate else 0) | (WP_HERMITIAN_PAIRS if hermitian_pairs else 0)
                 | (WP_KEEP_BINNING if keep_binning else 0) | (WP_COMPENSATED if compensated else 0))
        self._last_grid_shape = None
        self._check(lib.wp_grid(self._h, _ptr(uvw), _ptr(freq), _ptr(vis), _ptr(weight), nrow, nchan, flags,
                                _ptr(grid), _ptr(sum_w), _ptr(n_dropped), self._stream(stream)), "wp_grid")
        if keep_binning:
            self._last_grid_shape = (nrow, nchan)
        return grid, sum_w, n_dropped

    def degrid(self, uvw, freq, grid, vis_out=None, stream=None):
        import torch
        _dev_tensor(uvw, torch.float64, "uvw")
        _dev_tensor(freq, torch.float64, "freq")
        _dev_tensor(grid, torch.complex64, "grid", (self.n, self.n))
        nrow, nchan = uvw.shape[0], freq.shape[0]
        if vis_out is None:
            vis_out = torch.empty((nrow, nchan), dtype=torch.complex64, device=grid.device)
        _dev_tensor(vis_out, torch.complex64, "vis_out", (nrow, nchan))
        self._last_grid_shape = None
        self._check(lib.wp_degrid(self._h, _ptr(uvw), _ptr(freq), _ptr(grid), nrow, nchan, _ptr(vis_out),
                                  self._stream(stream)), "wp_degrid")
        return vis_out

    def degrid_last(self, grid, vis_out=None, stream=None):
        """Degrids the visibilities of the most recent grid(..., keep_binning=True) call, reusing its
        binning (wp_degrid_last)."""
        import torch
        _dev_tensor(grid, torch.complex64, "grid", (self.n, self.n))
        shape = getattr(self, "_last_grid_shape", None)
        if shape is None:
            raise WProjError(WP_ESTATE, "degrid_last: no grid() binning to reuse")
        if vis_out is None:
            vis_out = torch.empty(shape, dtype=torch.complex64, device=grid.device)
        _dev_tensor(vis_out, torch.complex64, "vis_out", shape)
        self._check(lib.wp_degrid_last(self._h, _ptr(grid), _ptr(vis_out), self._stream(stream)), "wp_degrid_last")
        return vis_out

    def fft_to_image(self, grid, sum_w, taper_correct: bool = True, image=None, stream=None):
        """Dirty image [N, N] float32. `grid` is clobbered (in-place FFT buffer)."""
        import torch
        _dev_tensor(grid, torch.complex64, "grid", (self.n, self.n))
        _dev_tensor(sum_w, torch.float64, "sum_w")
        if image is None:
            image = torch.empty((self.n, self.n), dtype=torch.float32, device=grid.device)
        _dev_tensor(image, torch.float32, "image", (self.n, self.n))
        self._check(lib.wp_fft_to_image(self._h, _ptr(grid), _ptr(sum_w), 1 if taper_correct else 0, _ptr(image),
                                        self._stream(stream)), "wp_fft_to_image")
        return image

    def image_to_grid(self, image, sum_w=None, taper_correct: bool = True, grid=None, stream=None):
        """Adjoint of fft_to_image: the [N, N] complex64 grid of a real [N, N] float32 image."""
        import torch
        _dev_tensor(image, torch.float32, "image", (self.n, self.n))
        if sum_w is not None:
            _dev_tensor(sum_w, torch.float64, "sum_w")
        if grid is None:
            grid = torch.empty((self.n, self.n), dtype=torch.complex64, device=image.device)
        _dev_tensor(grid, torch.complex64, "grid", (self.n, self.n))
        self._check(lib.wp_image_to_grid(self._h, _ptr(image), _ptr(sum_w), 1 if taper_correct else 0, _ptr(grid),
                                         self._stream(stream)), "wp_image_to_grid")
        return grid

    def baseline_order(self, ant1, ant2, n_ant: int, stream=None):
        """(perm [nrow] int32, start [N_ant (N_ant + 1)/2 + 1] uint32 as int32 storage): rows grouped
        by the baseline index of Eq. 5, time-ordered within each baseline; start holds Eq. 6."""
        import torch
        _dev_tensor(ant1, torch.int32, "ant1")
        nrow = ant1.shape[0]
        _dev_tensor(ant2, torch.int32, "ant2", (nrow,))
        nb = n_ant * (n_ant + 1) // 2
        perm = torch.empty(nrow, dtype=torch.int32, device=ant1.device)
        start = torch.empty(nb + 1, dtype=torch.int32, device=ant1.device)
        self._check(lib.wp_baseline_order(self._h, _ptr(ant1), _ptr(ant2), nrow, n_ant, _ptr(perm), _ptr(start),
                                          self._stream(stream)), "wp_baseline_order")
        return perm, start

    def grid_baseline(self, uvw, freq, vis, perm, start, n_ant: int, weight=None, grid=None, sum_w=None,
                      n_dropped=None, hermitian_pairs: bool = False, accumulate: bool = False, stream=None):
        """wp_grid's results through the paper's baseline-ordered kernel (perm, start from
        baseline_order)."""
        import torch
        dev = torch.device("cuda", self.device)
        _dev_tensor(uvw, torch.float64, "uvw")
        nrow = uvw.shape[0]
        _dev_tensor(freq, torch.float64, "freq")
        nchan = freq.shape[0]
        _dev_tensor(vis, torch.complex64, "vis", (nrow, nchan))
        _dev_tensor(perm, torch.int32, "perm", (nrow,))
        _dev_tensor(start, torch.int32, "start", (n_ant * (n_ant + 1) // 2 + 1,))
        if weight is not None:
            _dev_tensor(weight, torch.float32, "weight", (nrow, nchan))
        if grid is None:
            grid = torch.empty((self.n, self.n), dtype=torch.complex64, device=dev)
        _dev_tensor(grid, torch.complex64, "grid", (self.n, self.n))
        if sum_w is None:
            sum_w = torch.zeros(1, dtype=torch.float64, device=dev)
        if n_dropped is None:
            n_dropped = torch.zeros(1, dtype=torch.int64, device=dev)
        flags = (WP_ACCUMULATE if accumulate else 0) | (WP_HERMITIAN_PAIRS if hermitian_pairs else 0)
        self._check(lib.wp_grid_baseline(self._h, _ptr(uvw), _ptr(freq), _ptr(vis), _ptr(weight), _ptr(perm),
                                         _ptr(start), n_ant, nrow, nchan, flags, _ptr(grid), _ptr(sum_w),
                                         _ptr(n_dropped), self._stream(stream)), "wp_grid_baseline")
        return grid, sum_w, n_dropped

    def coords(self, uvw, freq, hermitian_pairs: bool = False, stream=None):
        """[ngridded, 8] int32: U, V, plane, conj, keep, i0, j0, ox | oy << 16."""
        import torch
        _dev_tensor(uvw, torch.float64, "uvw")
        _dev_tensor(freq, torch.float64, "freq")
        nrow, nchan = uvw.shape[0], freq.shape[0]
        ng = nrow * nchan * (2 if hermitian_pairs else 1)
        out = torch.empty((ng, 8), dtype=torch.int32, device=uvw.device)
        self._check(lib.wp_coords(self._h, _ptr(uvw), _ptr(freq), nrow, nchan,
                                  WP_HERMITIAN_PAIRS if hermitian_pairs else 0, _ptr(out), self._stream(stream)),
                    "wp_coords")
        return out

    def plane_info(self):
        sup = np.zeros(self.n_w, np.int32)
        w = np.zeros(self.n_w, np.float64)
        self._check(lib.wp_plane_info(self._h, sup.ctypes.data, w.ctypes.data), "wp_plane_info")
        return sup, w

    def wkernel_export(self, plane: int, stored: bool = False) -> np.ndarray:
        """Plane p's kernel [S os, S os] (canonical layout): float64 table or stored values."""
        sup, _ = self.plane_info()
        e = int(sup[plane]) * self.oversample
        out = np.zeros((e, e), np.complex128 if not stored else np.complex64)
        self._check(lib.wp_wkernel_export(self._h, plane, 1 if stored else 0, out.ctypes.data, e * e),
                    "wp_wkernel_export")
        return out

    def wkernel_norm(self) -> float:
        v = ctypes.c_double()
        self._check(lib.wp_wkernel_norm(self._h, ctypes.byref(v)), "wp_wkernel_norm")
        return v.value

    def profile(self, enable: bool = True):
        self._check(lib.wp_profile(self._h, 1 if enable else 0), "wp_profile")

    def profile_read(self) -> tuple[dict, dict, int]:
        """({phase: ms}, {phase: count}, own kernel launches) since the last read (synchronous)."""
        ms = np.zeros(len(PHASES), np.float64)
        cnt = np.zeros(len(PHASES), np.int32)
        nl = ctypes.c_int64()
        self._check(lib.wp_profile_read(self._h, ms.ctypes.data, cnt.ctypes.data, ctypes.byref(nl)),
                    "wp_profile_read")
        return dict(zip(PHASES, ms.tolist())), dict(zip(PHASES, cnt.tolist())), nl.value


class WBatch:
    """Many gridding jobs (each a WProj with its own geometry) gridded by wp_batch_grid: the jobs'
    coordinates and binning, then one persistent gridding launch over all of them.

    jobs: list of dicts with keys wp, uvw, freq, vis, and optionally weight, grid, sum_w,
    n_dropped, hermitian_pairs, accumulate. The tensors are fixed at creation (kept referenced
    here); their contents are read at every grid() call, so a captured graph can be replayed on
    new data written into the same tensors."""

    def __init__(self, jobs):
        import torch
        self._keep = []
        arr = (Job * len(jobs))()
        self.outputs = []
        for i, j in enumerate(jobs):
            wp = j["wp"]
            uvw, freq, vis = j["uvw"], j["freq"], j["vis"]
            _dev_tensor(uvw, torch.float64, "uvw")
            _dev_tensor(freq, torch.float64, "freq")
            nrow, nchan = uvw.shape[0], freq.shape[0]
            _dev_tensor(vis, torch.complex64, "vis", (nrow, nchan))
            weight = j.get("weight")
            if weight is not None:
                _dev_tensor(weight, torch.float32, "weight", (nrow, nchan))
            dev = uvw.device
            grid = j.get("grid")
            if grid is None:
                grid = torch.empty((wp.n, wp.n), dtype=torch.complex64, device=dev)
            _dev_tensor(grid, torch.complex64, "grid", (wp.n, wp.n))
            sum_w = j.get("sum_w")
            if sum_w is None:
                sum_w = torch.zeros(1, dtype=torch.float64, device=dev)
            nd = j.get("n_dropped")
            if nd is None:
                nd = torch.zeros(1, dtype=torch.int64, device=dev)
            flags = (WP_ACCUMULATE if j.get("accumulate") else 0) | (WP_HERMITIAN_PAIRS if j.get("hermitian_pairs") else 0)
            arr[i] = Job(wp._h, uvw.data_ptr(), freq.data_ptr(), vis.data_ptr(),
                         None if weight is None else weight.data_ptr(), nrow, nchan, flags, grid.data_ptr(),
                         sum_w.data_ptr(), nd.data_ptr())
            self._keep += [wp, uvw, freq, vis, weight, grid, sum_w, nd]
            self.outputs.append((grid, sum_w, nd))
        h = ctypes.c_void_p()
        rc = lib.wp_batch_create(arr, len(jobs), ctypes.byref(h))
        if rc != WP_OK:
            msg = ""
            for j in jobs:
                m = lib.wp_last_error(j["wp"]._h)
                if m:
                    msg = m.decode()
            raise WProjError(rc, f"wp_batch_create: {msg}")
        self._h = h
        self._jobs = arr

    @property
    def fused_jobs(self) -> int:
        return int(lib.wp_batch_fused_jobs(self._h))

    def grid(self, stream=None):
        import torch
        s = torch.cuda.current_stream() if stream is None else stream
        rc = lib.wp_batch_grid(self._h, ctypes.c_void_p(s.cuda_stream))
        if rc != WP_OK:
            raise WProjError(rc, "wp_batch_grid")
        return self.outputs

    def capture(self):
        """A torch.cuda.CUDAGraph replaying grid() (one eager run first warms every buffer)."""
        import torch
        self.grid()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.grid()
        return g

    def close(self):
        if getattr(self, "_h", None):
            lib.wp_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
