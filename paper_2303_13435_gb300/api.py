"""ctypes binding of libur (include/ur.h): argument marshalling only.

Every computation runs in the CUDA library; PyTorch supplies device memory,
pinned host memory and streams.  Loading fails loudly when libur.so is absent:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libur.so")

UR_F32, UR_F16 = 0, 1
UR_WS_FORWARD, UR_WS_BACKWARD, UR_WS_HOST_SLABS, UR_WS_ADJ_SLABS = 1, 2, 4, 8
BIN_FIELDS = 6
BIN_COUNT, BIN_SUM_I, BIN_SUM_I2, BIN_SUM_Q, BIN_MEAN, BIN_SEM = range(6)
STATUS = {0: "UR_OK", 1: "UR_ERR_INVALID", 2: "UR_ERR_OOM", 3: "UR_ERR_CUDA", 4: "UR_ERR_TIMEOUT",
          5: "UR_ERR_UNSUPPORTED", 6: "UR_ERR_FAULT_INJECTED"}

# exported symbols of include/ur.h, with (restype, argtypes)
_vp, _i32, _i64, _sz, _dp = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t, C.POINTER(C.c_double)


class GridDesc(C.Structure):
    _fields_ = [("n", C.c_int32), ("dx", C.c_double), ("ed_dtype", C.c_int32), ("z0", C.c_int32), ("nz", C.c_int32)]


class ShapeDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("center", C.c_float * 3), ("size", C.c_float), ("rot", C.c_float * 9)]


class LatticeDesc(C.Structure):
    _fields_ = [("rot", C.c_float * 9), ("offset", C.c_float * 3)]


def lattice_desc(lattice) -> LatticeDesc:
    """(R, q) -> ur_lattice: sample point p = R (x - c) + q in cell-voxel units."""
    rot, off = lattice
    d = LatticeDesc()
    r = np.asarray(rot, dtype=np.float32).reshape(9)
    for i in range(9):
        d.rot[i] = float(r[i])
    o = np.asarray(off, dtype=np.float32)
    for i in range(3):
        d.offset[i] = float(o[i])
    return d


class DetectorDesc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("pixel_m", C.c_double), ("distance_m", C.c_double),
                ("beam_x", C.c_double), ("beam_y", C.c_double), ("wavelength_nm", C.c_double),
                ("bandwidth", C.c_double), ("nlambda", C.c_int32), ("rot", C.c_float * 9)]


class BatchItem(C.Structure):
    _fields_ = [("plan", C.c_void_p), ("cell", C.c_void_p), ("ucell", C.c_int32), ("origin", C.c_int32 * 3),
                ("shape", ShapeDesc), ("weights", C.c_void_p), ("bins", C.c_void_p), ("ws", C.c_void_p),
                ("ws_bytes", C.c_size_t), ("dl_dmean", C.c_void_p), ("dl_dcell", C.c_void_p),
                ("dl_dmask", C.c_void_p)]


SIGNATURES = {
    "ur_last_error": (C.c_char_p, []),
    "ur_version": (C.c_char_p, []),
    "ur_plan_create": (_i32, [C.POINTER(GridDesc), _dp, _i32, C.POINTER(_vp)]),
    "ur_plan_destroy": (_i32, [_vp]),
    "ur_plan_thresholds": (_i32, [_vp, C.POINTER(C.c_int64)]),
    "ur_bin_thresholds": (_i32, [_i32, C.c_double, _dp, _i32, C.POINTER(C.c_int64)]),
    "ur_fault_reset": (None, []),
    "ur_workspace_size": (_sz, [_vp, _i32]),
    "ur_plan_set_slab_planes": (_i32, [_vp, _i32]),
    "ur_build_density": (_i32, [_i32, _vp, _i32, C.POINTER(C.c_int32), C.POINTER(ShapeDesc), _vp, _i32, _i32, _i32,
                                _vp, _vp, _vp]),
    "ur_build_density_lattice": (_i32, [_i32, _vp, _i32, C.POINTER(LatticeDesc), C.POINTER(ShapeDesc), _vp, _i32, _i32,
                                        _i32, _vp, _vp, _vp]),
    "ur_zoom_density": (_i32, [_i32, _i32, _vp, _i32, _i32, _i32, _vp, _vp]),
    "ur_fft_intensity": (_i32, [_vp, _vp, _i32, _vp, _vp, _vp, _sz, _vp]),
    "ur_fft_intensity_tiled": (_i32, [_vp, _vp, _i32, C.POINTER(C.c_int32), C.POINTER(ShapeDesc), _vp, _vp, _vp, _vp,
                                      _sz, _vp]),
    "ur_fft_intensity_tiled_lattice": (_i32, [_vp, _vp, _i32, C.POINTER(LatticeDesc), C.POINTER(ShapeDesc), _vp, _vp,
                                              _vp, _vp, _sz, _vp]),
    "ur_fft_intensity_noalloc": (_i32, [_vp, _vp, _vp, _vp]),
    "ur_noalloc_scratch_bytes": (_sz, []),
    "ur_bin_q": (_i32, [_vp, _vp, _vp, _vp, _sz, _vp]),
    "ur_merge": (_i32, [_i32, C.POINTER(_vp), C.POINTER(C.c_int32), _dp, _vp, _i32, _i32, _vp, _vp]),
    "ur_level_qmax": (C.c_double, [C.c_double]),
    "ur_ewald_image": (_i32, [_vp, _vp, C.POINTER(DetectorDesc), _vp, _vp]),
    "ur_ensemble": (_i32, [_i32, C.POINTER(_vp), C.POINTER(C.c_int32), _dp, _i32, _vp, _vp]),
    "ur_ensemble_backward": (_i32, [_i32, C.POINTER(_vp), C.POINTER(C.c_int32), _dp, _i32, _vp, C.POINTER(_vp), _vp]),
    "ur_backward": (_i32, [_vp, _vp, _vp, _vp, _vp, _i32, C.POINTER(C.c_int32), C.POINTER(ShapeDesc), _vp, _vp, _vp,
                           _vp, _sz, _vp]),
    "ur_backward_slabs": (_i32, [_vp, _vp, _vp, _vp, _i32, C.POINTER(C.c_int32), C.POINTER(ShapeDesc), _vp, _vp, _vp,
                                 _vp, _sz, _vp]),
    "ur_plan_set_adj_slab_planes": (_i32, [_vp, _i32]),
    "ur_set_timing": (None, [_i32]),
    "ur_last_timings": (_i32, [C.POINTER(C.c_float), _i32, C.POINTER(C.c_char_p)]),
    "ur_batch_create": (_i32, [_i32, _vp, C.POINTER(_vp)]),
    "ur_batch_destroy": (_i32, [_vp]),
    "ur_batch_forward": (_i32, [_vp, _vp]),
    "ur_batch_backward": (_i32, [_vp, _vp]),
    "ur_plan_set_tiles": (_i32, [_vp, _i32, _i32]),
    "ur_plan_set_chunk_planes": (_i32, [_vp, _i32]),
    "ur_sync_status": (_i32, [_vp]),
    "ur_log_mse_grad": (_i32, [_i32, _vp, _vp, _vp, _vp, _vp]),
    "ur_plan_chunk_planes": (_i32, [_vp]),
    "ur_plan_get_tiles": (_i32, [_vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "ur_plan_set_voxel_sinc": (_i32, [_vp, _i32]),
    "ur_plan_set_tma_zpass": (_i32, [_vp, _i32]),
    "ur_plan_tma_zpass": (_i32, [_vp]),
    "ur_plan_voxel_sinc": (_i32, [_vp]),
}
# test hooks (not part of the header's API)
EXTRA = {
    "ur_selftest_fastdiv": (C.c_int64, []),
    "ur_selftest_dft": (C.c_double, []),
    "ur_selftest_wait_timeout": (_i32, [_vp]),
}

_lib = None


class UrError(RuntimeError):
    def __init__(self, fn: str, status: int, msg: str):
        super().__init__(f"{fn} -> {STATUS.get(status, status)}: {msg}")
        self.status = status


def lib() -> C.CDLL:
    """Load libur.so (built by paper_2303_13435_gb300.build); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libur.so not found at {LIB_PATH}: run __graft_entry__.build() first")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in {**SIGNATURES, **EXTRA}.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(fn: str, st: int):
    if st != 0:
        raise UrError(fn, st, lib().ur_last_error().decode(errors="replace"))


def _ptr(t) -> int | None:
    if t is None:
        return None
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _dtype_code(d) -> int:
    if d in ("f32", torch.float32, np.float32):
        return UR_F32
    if d in ("f16", torch.float16, np.float16):
        return UR_F16
    raise ValueError(f"unsupported ED dtype {d}")


def _torch_dtype(code: int):
    return torch.float32 if code == UR_F32 else torch.float16


def shape_desc(shape) -> ShapeDesc:
    d = ShapeDesc()
    d.kind = int(shape.kind)
    c = np.asarray(shape.center, dtype=np.float32)
    for i in range(3):
        d.center[i] = float(c[i])
    d.size = float(np.float32(shape.size))
    r = np.asarray(shape.rot, dtype=np.float32).reshape(9)
    for i in range(9):
        d.rot[i] = float(r[i])
    return d


class Plan:
    """ur_plan: grid, ED storage type, the nonzero plane slab [z0, z0+nz) and the Q bins."""

    def __init__(self, n: int, dx: float, edges, z0: int = 0, nz: int | None = None, ed_dtype="f32"):
        self.n = int(n)
        self.dx = float(dx)
        self.edges = np.ascontiguousarray(edges, dtype=np.float64)
        self.nbins = len(self.edges) - 1
        self.z0 = int(z0)
        self.nz = int(self.n - z0 if nz is None else nz)
        self.ed_dtype = _dtype_code(ed_dtype)
        g = GridDesc(self.n, self.dx, self.ed_dtype, self.z0, self.nz)
        h = C.c_void_p()
        _check("ur_plan_create", lib().ur_plan_create(C.byref(g), self.edges.ctypes.data_as(_dp), self.nbins, C.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def thresholds(self) -> np.ndarray:
        out = np.zeros(self.nbins + 1, dtype=np.int64)
        _check("ur_plan_thresholds", lib().ur_plan_thresholds(self._h, out.ctypes.data_as(C.POINTER(C.c_int64))))
        return out

    def workspace_size(self, what: int = UR_WS_FORWARD) -> int:
        return int(lib().ur_workspace_size(self._h, what))

    def set_tiles(self, rows_per_block: int = 0, cols_per_block: int = 0):
        _check("ur_plan_set_tiles", lib().ur_plan_set_tiles(self._h, int(rows_per_block), int(cols_per_block)))

    def tiles(self) -> tuple[int, int]:
        r, c = C.c_int32(), C.c_int32()
        _check("ur_plan_get_tiles", lib().ur_plan_get_tiles(self._h, C.byref(r), C.byref(c)))
        return r.value, c.value

    def set_slab_planes(self, planes: int):
        _check("ur_plan_set_slab_planes", lib().ur_plan_set_slab_planes(self._h, int(planes)))

    def set_adj_slab_planes(self, planes: int):
        _check("ur_plan_set_adj_slab_planes", lib().ur_plan_set_adj_slab_planes(self._h, int(planes)))

    def set_chunk_planes(self, planes: int):
        _check("ur_plan_set_chunk_planes", lib().ur_plan_set_chunk_planes(self._h, int(planes)))

    def set_voxel_sinc(self, on: bool = True):
        """Bin |F|^2 times the voxel form factor prod_a sinc^2(pi k_a / N) (Sec. 2.5 sinc correction)."""
        _check("ur_plan_set_voxel_sinc", lib().ur_plan_set_voxel_sinc(self._h, 1 if on else 0))

    def set_tma_zpass(self, on: bool = True):
        """Select the TMA-staged z-pass engine (N = 256, 512) instead of the compile-time kernel."""
        _check("ur_plan_set_tma_zpass", lib().ur_plan_set_tma_zpass(self._h, 1 if on else 0))

    def tma_zpass(self) -> bool:
        return bool(lib().ur_plan_tma_zpass(self._h))

    def voxel_sinc(self) -> bool:
        return bool(lib().ur_plan_voxel_sinc(self._h))

    def chunk_planes(self) -> int:
        return int(lib().ur_plan_chunk_planes(self._h))

    def workspace(self, what: int = UR_WS_FORWARD, device="cuda") -> torch.Tensor:
        return torch.empty(self.workspace_size(what), dtype=torch.uint8, device=device)

    def claim_workspace(self, what: int = UR_WS_FORWARD, device="cuda") -> tuple[torch.Tensor, int]:
        """The plan's own workspace, allocated once (grown when `what` needs more) and reused by
        every claim.  Returns (workspace, generation); the generation changes at each claim, so
        a holder can tell whether someone else has written the workspace since its claim."""
        need = self.workspace_size(what)
        ws = getattr(self, "_ws", None)
        if ws is None or ws.numel() < need or ws.device != torch.device(device):
            ws = torch.empty(need, dtype=torch.uint8, device=device)
            self._ws = ws
        self._ws_gen = getattr(self, "_ws_gen", 0) + 1
        return ws, self._ws_gen

    def workspace_generation(self) -> int:
        return getattr(self, "_ws_gen", 0)

    def close(self):
        if getattr(self, "_h", None):
            lib().ur_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build_density(n: int, cell: torch.Tensor, shape, origin=(0, 0, 0), weights: torch.Tensor | None = None,
                  z_begin: int = 0, z_count: int | None = None, out_dtype="f32", out: torch.Tensor | None = None,
                  nz_range: torch.Tensor | None = None, lattice=None, stream=None) -> torch.Tensor:
    """ED-1 planes [z_begin, z_begin + z_count) (Sec. 2.3 tile + mask); lattice = (R, q) samples the
    cell on a rotated lattice instead of the integer wrap with `origin`."""
    z_count = n - z_begin if z_count is None else z_count
    code = _dtype_code(out_dtype)
    if out is None:
        out = torch.empty((z_count, n, n), dtype=_torch_dtype(code), device=cell.device)
    assert cell.is_cuda and cell.dtype == torch.float32 and cell.is_contiguous()
    sd = shape_desc(shape)
    if lattice is not None:
        ld = lattice_desc(lattice)
        _check("ur_build_density_lattice", lib().ur_build_density_lattice(
            n, _ptr(cell), cell.shape[0], C.byref(ld), C.byref(sd), _ptr(weights), z_begin, z_count, code, _ptr(out),
            _ptr(nz_range), _stream(stream)))
        return out
    org = (C.c_int32 * 3)(*[int(v) for v in origin])
    _check("ur_build_density", lib().ur_build_density(n, _ptr(cell), cell.shape[0], org, C.byref(sd), _ptr(weights),
                                                      z_begin, z_count, code, _ptr(out), _ptr(nz_range), _stream(stream)))
    return out


def zoom_density(src: torch.Tensor, f: int, n_out: int, out_dtype="f16", out: torch.Tensor | None = None,
                 stream=None) -> torch.Tensor:
    """ED-2/ED-3 (Sec. 2.3 block integration + zero padding)."""
    code = _dtype_code(out_dtype)
    if out is None:
        out = torch.empty((n_out, n_out, n_out), dtype=_torch_dtype(code), device=src.device)
    _check("ur_zoom_density", lib().ur_zoom_density(src.shape[0], _dtype_code(src.dtype), _ptr(src), f, n_out, code,
                                                    _ptr(out), _stream(stream)))
    return out


def new_bins(plan: Plan, device="cuda") -> torch.Tensor:
    return torch.empty((BIN_FIELDS, plan.nbins), dtype=torch.float64, device=device)


def fft_intensity(plan: Plan, ed: torch.Tensor, bins: torch.Tensor | None = None, F_out: torch.Tensor | None = None,
                  ws: torch.Tensor | None = None, stream=None, want_bins: bool = True):
    """Sec. 2.4-2.5: transform of the nz planes in `ed`, |F|^2 and Q-bin statistics.

    `ed` holds planes [z0, z0+nz) (device, or pinned host for the streamed path).
    Returns the bins tensor [6, B] (count, sum I, sum I^2, sum |Q|, mean, sem)."""
    on_host = 0 if ed.is_cuda else 1
    what = UR_WS_FORWARD | (UR_WS_HOST_SLABS if on_host else 0)
    if ws is None:
        ws = plan.workspace(what)
    if bins is None and want_bins:
        bins = new_bins(plan)
    _check("ur_fft_intensity", lib().ur_fft_intensity(plan.handle, _ptr(ed), on_host, _ptr(bins), _ptr(F_out), _ptr(ws),
                                                      ws.numel(), _stream(stream)))
    return bins


def fft_intensity_tiled(plan: Plan, cell: torch.Tensor, shape, origin=(0, 0, 0), weights: torch.Tensor | None = None,
                        bins: torch.Tensor | None = None, F_out: torch.Tensor | None = None,
                        ws: torch.Tensor | None = None, stream=None, want_bins: bool = True, lattice=None):
    """Sec. 2.3 + 2.4 + 2.5 fused: density generated inside the plane pass, never stored."""
    if ws is None:
        ws = plan.workspace(UR_WS_FORWARD)
    if bins is None and want_bins:
        bins = new_bins(plan)
    sd = shape_desc(shape)
    if lattice is not None:
        ld = lattice_desc(lattice)
        _check("ur_fft_intensity_tiled_lattice", lib().ur_fft_intensity_tiled_lattice(
            plan.handle, _ptr(cell), cell.shape[0], C.byref(ld), C.byref(sd), _ptr(weights), _ptr(bins), _ptr(F_out),
            _ptr(ws), ws.numel(), _stream(stream)))
        return bins
    org = (C.c_int32 * 3)(*[int(v) for v in origin])
    _check("ur_fft_intensity_tiled", lib().ur_fft_intensity_tiled(plan.handle, _ptr(cell), cell.shape[0], org,
                                                                  C.byref(sd), _ptr(weights), _ptr(bins), _ptr(F_out),
                                                                  _ptr(ws), ws.numel(), _stream(stream)))
    return bins


def log_mse_grad(bins: torch.Tensor, target: torch.Tensor, dl_dmean: torch.Tensor | None = None,
                 loss: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """dL/d(mean) of the log-I(Q) MSE against `target` (and L into `loss`, a device double[1])."""
    nb = bins.shape[1]
    assert bins.dtype == torch.float64 and target.dtype == torch.float64 and target.numel() == nb
    if dl_dmean is None:
        dl_dmean = torch.empty(nb, dtype=torch.float64, device=bins.device)
    _check("ur_log_mse_grad", lib().ur_log_mse_grad(nb, _ptr(bins), _ptr(target), _ptr(loss), _ptr(dl_dmean),
                                                    _stream(stream)))
    return dl_dmean


def sync_status(stream=None) -> None:
    """Wait for the work queued on `stream`; raises UrError if it failed on the device."""
    _check("ur_sync_status", lib().ur_sync_status(_stream(stream)))


def noalloc_scratch_bytes() -> int:
    """Size of the library's built-in scratch array used by fft_intensity_noalloc."""
    return int(lib().ur_noalloc_scratch_bytes())


def fft_intensity_noalloc(plan: Plan, ed: torch.Tensor, bins: torch.Tensor, stream=None) -> torch.Tensor:
    """ur_fft_intensity without a workspace, for callers that must not allocate while
    running: the intermediate sits in the library's built-in scratch array (noalloc_scratch_bytes()).
    `bins` must be preallocated by the caller; calls that overlap on the GPU race."""
    _check("ur_fft_intensity_noalloc", lib().ur_fft_intensity_noalloc(plan.handle, _ptr(ed), _ptr(bins),
                                                                      _stream(stream)))
    return bins


def bin_q(plan: Plan, I_half: torch.Tensor, bins: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    if bins is None:
        bins = new_bins(plan)
    _check("ur_bin_q", lib().ur_bin_q(plan.handle, _ptr(I_half), _ptr(bins), None, 0, _stream(stream)))
    return bins


MERGE_MODES = {"windows": 0, "invvar": 1}


def merge(level_bins: list, level_n: list, level_dx: list, edges_dev: torch.Tensor, out: torch.Tensor | None = None,
          mode: str = "windows", stream=None) -> torch.Tensor:
    """Sec. 2.5 merge of level curves into absolute units; out[5, B] = mean, sem, count, mean Q, source.

    level_dx: voxel edge of each level (nm); the library derives each level's limit from it."""
    nlev = len(level_bins)
    nb = edges_dev.numel() - 1
    if out is None:
        out = torch.empty((5, nb), dtype=torch.float64, device=edges_dev.device)
    ptrs = (C.c_void_p * nlev)(*[b.data_ptr() for b in level_bins])
    ns = (C.c_int32 * nlev)(*[int(v) for v in level_n])
    dxs = (C.c_double * nlev)(*[float(v) for v in level_dx])
    _check("ur_merge", lib().ur_merge(nlev, ptrs, ns, dxs, _ptr(edges_dev), nb, MERGE_MODES[mode], _ptr(out),
                                      _stream(stream)))
    return out


def ensemble(item_bins: list, item_n: list, weights, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Sec. 3 polydisperse ensemble: out[4, B] = mean (sum_i w_i N_i^6 mean_i), SEM, count, mean Q."""
    k = len(item_bins)
    nb = item_bins[0].shape[1]
    if out is None:
        out = torch.empty((4, nb), dtype=torch.float64, device=item_bins[0].device)
    ptrs = (C.c_void_p * k)(*[b.data_ptr() for b in item_bins])
    ns = (C.c_int32 * k)(*[int(v) for v in item_n])
    ws = np.ascontiguousarray(weights, dtype=np.float64)
    _check("ur_ensemble", lib().ur_ensemble(k, ptrs, ns, ws.ctypes.data_as(_dp), nb, _ptr(out), _stream(stream)))
    return out


def ensemble_backward(item_bins: list, item_n: list, weights, dl_dens: torch.Tensor, item_dl_dmean: list,
                      stream=None):
    """dL/d(each particle's bin means) from dL/d(ensemble mean) (written into item_dl_dmean)."""
    k = len(item_bins)
    nb = item_bins[0].shape[1]
    ptrs = (C.c_void_p * k)(*[b.data_ptr() for b in item_bins])
    gp = (C.c_void_p * k)(*[g.data_ptr() for g in item_dl_dmean])
    ns = (C.c_int32 * k)(*[int(v) for v in item_n])
    ws = np.ascontiguousarray(weights, dtype=np.float64)
    _check("ur_ensemble_backward", lib().ur_ensemble_backward(k, ptrs, ns, ws.ctypes.data_as(_dp), nb, _ptr(dl_dens),
                                                              gp, _stream(stream)))
    return item_dl_dmean


def ewald_image(plan: Plan, F_half: torch.Tensor, det: dict, out: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
    """Sec. 2.5 detector image on the Ewald sphere from the half spectrum F (F_out of a forward).
    det: nx, ny, pixel_m, distance_m, beam (bx, by), wavelength_nm, bandwidth, nlambda, rot."""
    d = DetectorDesc()
    d.nx, d.ny = int(det["nx"]), int(det["ny"])
    d.pixel_m, d.distance_m = float(det["pixel_m"]), float(det["distance_m"])
    d.beam_x, d.beam_y = float(det["beam"][0]), float(det["beam"][1])
    d.wavelength_nm, d.bandwidth = float(det["wavelength_nm"]), float(det.get("bandwidth", 0.0))
    d.nlambda = int(det.get("nlambda", 1))
    r = np.asarray(det.get("rot", np.eye(3)), dtype=np.float32).reshape(9)
    for i in range(9):
        d.rot[i] = float(r[i])
    if out is None:
        out = torch.empty((d.ny, d.nx), dtype=torch.float32, device=F_half.device)
    _check("ur_ewald_image", lib().ur_ewald_image(plan.handle, _ptr(F_half), C.byref(d), _ptr(out), _stream(stream)))
    return out


def level_qmax(dx: float) -> float:
    """The |Q| up to which ur_merge trusts a level of voxel edge dx (computed by the library)."""
    return float(lib().ur_level_qmax(float(dx)))


def backward(plan: Plan, dl_dmean: torch.Tensor, fwd_bins: torch.Tensor, cell: torch.Tensor, shape, ws: torch.Tensor,
             origin=(0, 0, 0), weights: torch.Tensor | None = None, F: torch.Tensor | None = None,
             dl_dcell: torch.Tensor | None = None, dl_dmask: torch.Tensor | None = None, want_mask: bool = True,
             stream=None):
    """Adjoint: dL/d(mean I) -> (dL/d cell, dL/d mask).  `ws` is the forward's workspace
    (sized UR_WS_FORWARD | UR_WS_BACKWARD) still holding the forward intermediate."""
    n = plan.n
    if dl_dcell is None:
        dl_dcell = torch.empty_like(cell)
    if dl_dmask is None and want_mask:
        dl_dmask = torch.empty((n, n, n), dtype=torch.float32, device=cell.device)
    org = (C.c_int32 * 3)(*[int(v) for v in origin])
    sd = shape_desc(shape)
    _check("ur_backward", lib().ur_backward(plan.handle, _ptr(dl_dmean), _ptr(fwd_bins), _ptr(F), _ptr(cell),
                                            cell.shape[0], org, C.byref(sd), _ptr(weights), _ptr(dl_dcell),
                                            _ptr(dl_dmask), _ptr(ws), ws.numel(), _stream(stream)))
    return dl_dcell, dl_dmask


def backward_slabs(plan: Plan, dl_dmean: torch.Tensor, fwd_bins: torch.Tensor, cell: torch.Tensor, shape,
                   ws: torch.Tensor, origin=(0, 0, 0), weights: torch.Tensor | None = None,
                   dl_dcell: torch.Tensor | None = None, dl_dmask_host: torch.Tensor | None = None, stream=None):
    """Out-of-core adjoint: dL/d cell on the device, dL/d mask (optional) into pinned host memory,
    slab by slab with the z pass recomputed per slab.  `ws` (UR_WS_FORWARD | UR_WS_ADJ_SLABS) still
    holds the forward intermediate."""
    if dl_dcell is None:
        dl_dcell = torch.empty_like(cell)
    org = (C.c_int32 * 3)(*[int(v) for v in origin])
    sd = shape_desc(shape)
    _check("ur_backward_slabs", lib().ur_backward_slabs(plan.handle, _ptr(dl_dmean), _ptr(fwd_bins), _ptr(cell),
                                                        cell.shape[0], org, C.byref(sd), _ptr(weights),
                                                        _ptr(dl_dcell), _ptr(dl_dmask_host), _ptr(ws), ws.numel(),
                                                        _stream(stream)))
    return dl_dcell, dl_dmask_host


def bin_thresholds(n: int, dx: float, edges) -> np.ndarray:
    """Integer k^2 thresholds of the bins (host computation, no GPU)."""
    e = np.ascontiguousarray(edges, dtype=np.float64)
    out = np.zeros(len(e), dtype=np.int64)
    _check("ur_bin_thresholds", lib().ur_bin_thresholds(n, dx, e.ctypes.data_as(_dp), len(e) - 1,
                                                        out.ctypes.data_as(C.POINTER(C.c_int64))))
    return out


class Batch:
    """ur_batch over particles of uneven grids: one forward and one adjoint launch
    sequence for all of them.  Each particle: a Plan, the cell (device float32
    U^3), a Shape, and optional adjoint buffers; the batch allocates (via torch)
    each particle's bins, workspace, dL/dmean input and dL/d cell output."""

    def __init__(self, plans, cells, shapes, origins=None, with_backward=True, with_mask_grad=False):
        self.plans = list(plans)
        n = len(self.plans)
        self.cells = list(cells) if isinstance(cells, (list, tuple)) else [cells] * n
        self.shapes = list(shapes)
        origins = origins or [(0, 0, 0)] * n
        what = UR_WS_FORWARD | (UR_WS_BACKWARD if with_backward else 0)
        self.bins = [new_bins(p) for p in self.plans]
        self.ws = [p.workspace(what) for p in self.plans]
        self.dl_dmean = [torch.zeros(p.nbins, dtype=torch.float64, device="cuda") if with_backward else None
                         for p in self.plans]
        self.dl_dcell = [torch.zeros_like(c) if with_backward else None for c in self.cells]
        self.dl_dmask = [torch.zeros((p.n, p.n, p.n), dtype=torch.float32, device="cuda")
                         if (with_backward and with_mask_grad) else None for p in self.plans]
        items = (BatchItem * n)()
        for i in range(n):
            it = items[i]
            it.plan = self.plans[i].handle.value
            it.cell = self.cells[i].data_ptr()
            it.ucell = self.cells[i].shape[0]
            for a in range(3):
                it.origin[a] = int(origins[i][a])
            it.shape = shape_desc(self.shapes[i])
            it.weights = None
            it.bins = self.bins[i].data_ptr()
            it.ws = self.ws[i].data_ptr()
            it.ws_bytes = self.ws[i].numel()
            it.dl_dmean = self.dl_dmean[i].data_ptr() if with_backward else None
            it.dl_dcell = self.dl_dcell[i].data_ptr() if with_backward else None
            it.dl_dmask = self.dl_dmask[i].data_ptr() if self.dl_dmask[i] is not None else None
        h = C.c_void_p()
        _check("ur_batch_create", lib().ur_batch_create(n, C.cast(items, C.c_void_p), C.byref(h)))
        self._h = h

    def forward(self, stream=None):
        _check("ur_batch_forward", lib().ur_batch_forward(self._h, _stream(stream)))
        return self.bins

    def backward(self, stream=None):
        _check("ur_batch_backward", lib().ur_batch_backward(self._h, _stream(stream)))
        return self.dl_dcell

    def close(self):
        if getattr(self, "_h", None):
            lib().ur_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def set_timing(enable: bool):
    lib().ur_set_timing(1 if enable else 0)


def last_timings(max_entries: int = 4096):
    ms = (C.c_float * max_entries)()
    names = (C.c_char_p * max_entries)()
    n = lib().ur_last_timings(ms, max_entries, names)
    return [(names[i].decode(), float(ms[i])) for i in range(n)]


def header_symbols() -> list[str]:
    """Function names declared in include/ur.h."""
    import re
    hdr = os.path.join(os.path.dirname(HERE), "include", "ur.h")
    txt = open(hdr).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ur_[a-z0-9_]+)\s*\(", txt)))

