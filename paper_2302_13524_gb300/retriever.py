"""Retriever: one TM retrieval problem on the GPU, as torch tensors in and out.

A thin owner of a libtmr handle (tmr_create): it checks that every input is a
contiguous tensor of the right dtype and shape on the handle's device,
allocates the outputs there, and calls the C entry points of the same names.
All arithmetic runs in libtmr's kernels.
"""
from __future__ import annotations

import torch

from . import _lib

_DT = {"c64": torch.complex64, "f32": torch.float32, "f64": torch.float64, "i32": torch.int32}


class Retriever:
    """Retrieve an M x N transmission matrix from J masked-DFT intensity sets
    (Algorithm 1 per row, then the defocus phase-offset fit).

    masks: complex64 tensor [J, N] (|d| = 1).  defocus: None,
    dict(ny, nx, n_defocus, coef=0.05, H=None) (same-grid operator, images
    [n_defocus, M]) or dict(kind=1, ny, nx, n_defocus, wavelength, na, z_d,
    pixel, incident) (angular spectrum with 2x padding, images
    [n_defocus, 4 M] on the 2ny x 2nx grid).  options: the fields of
    tmr_options (m, init, seed, power_iters, clip, tol, phase_iters, precision,
    use_graph, workspace_limit, schedule, tune_cache).
    """

    def __init__(self, masks: torch.Tensor, M: int, defocus=None, stream: torch.cuda.Stream | None = None,
                 **options):
        if not isinstance(masks, torch.Tensor) or not masks.is_cuda:
            raise TypeError("masks: a CUDA tensor is expected")
        J, N = masks.shape
        self.device = masks.device
        self.N, self.M, self.J = int(N), int(M), int(J)
        self.stream = stream
        self.h = _lib.tmr_create(self.N, self.M, self.J, self._check(masks, "c64", (J, N), "masks"),
                                 defocus, options or None,
                                 stream=stream.cuda_stream if stream is not None else None)

    # -- argument checks ---------------------------------------------------
    def _check(self, x, dt, shape, name):
        if not isinstance(x, torch.Tensor):
            raise TypeError(f"{name}: a torch tensor is expected")
        if x.device != self.device:
            raise ValueError(f"{name}: on {x.device}, the handle is on {self.device}")
        if x.dtype != _DT[dt]:
            raise TypeError(f"{name}: dtype {x.dtype}, expected {_DT[dt]}")
        if tuple(x.shape) != tuple(shape):
            raise ValueError(f"{name}: shape {tuple(x.shape)}, expected {tuple(shape)}")
        if not x.is_contiguous():
            raise ValueError(f"{name}: not contiguous")
        return x

    def _empty(self, shape, dt):
        return torch.empty(shape, dtype=_DT[dt], device=self.device)

    # -- the C entry points ------------------------------------------------
    def forward(self, T: torch.Tensor) -> torch.Tensor:
        """Y[r, j, k] = |F(d_j .* T[r])[k]|^2 (Eq. optTMsmall2)."""
        Y = self._empty((self.M, self.J, self.N), "f32")
        _lib.tmr_forward(self.h, self._check(T, "c64", (self.M, self.N), "T"), Y)
        return Y

    def grad(self, T: torch.Tensor, Y: torch.Tensor):
        """(loss [M], gradient [M, N]) of f(t) = ||y - |Q t|^2||^2 per row (Eq. derivative)."""
        loss = self._empty((self.M,), "f32")
        G = self._empty((self.M, self.N), "c64")
        _lib.tmr_grad(self.h, self._check(T, "c64", (self.M, self.N), "T"),
                      self._check(Y, "f32", (self.M, self.J, self.N), "Y"), loss, G)
        return loss, G

    def retrieve(self, y: torch.Tensor, y_def: torch.Tensor | None = None, iters: int = 100,
                 T_init: torch.Tensor | None = None) -> dict:
        """The whole path; returns dict(T, status, iters, loss) (tensors on the device)."""
        out = dict(T=self._empty((self.M, self.N), "c64"), status=self._empty((self.M,), "i32"),
                   iters=self._empty((self.M,), "i32"), loss=self._empty((self.M,), "f32"))
        y = self._check(y, "f32", (self.M, self.J, self.N), "y")
        if y_def is not None:
            y_def = self._check(y_def, "f32", (self.h.n_defocus, self.h.defocus_pixels), "y_def")
        if T_init is None:
            _lib.tmr_retrieve(self.h, y, y_def, iters, out["T"], out["status"], out["iters"], out["loss"])
        else:
            _lib.tmr_retrieve_from(self.h, self._check(T_init, "c64", (self.M, self.N), "T_init"), y, y_def,
                                   iters, out["T"], out["status"], out["iters"], out["loss"])
        return out

    def defocus_forward(self, T: torch.Tensor) -> torch.Tensor:
        """Defocus-plane intensities [n_defocus, M] (kind 0) or [n_defocus, 4 M] (kind 1) (Eq. forwarddefocusImage)."""
        Yd = self._empty((self.h.n_defocus, self.h.defocus_pixels), "f32")
        _lib.tmr_defocus_forward(self.h, self._check(T, "c64", (self.M, self.N), "T"), Yd)
        return Yd

    def defocus_fit(self, T_est: torch.Tensor, y_def: torch.Tensor):
        """(phi [M] float64, diag(e^{i phi}) T_est) from the defocus fit (Eq. optphase)."""
        phi = self._empty((self.M,), "f64")
        T = self._empty((self.M, self.N), "c64")
        _lib.tmr_defocus_fit(self.h, self._check(T_est, "c64", (self.M, self.N), "T_est"),
                             self._check(y_def, "f32", (self.h.n_defocus, self.h.defocus_pixels), "y_def"), phi, T)
        return phi, T

    def sync(self, timeout_s: float = 60.0):
        _lib.tmr_sync(self.h, timeout_s)

    @property
    def schedule(self) -> int:
        """Masks per CTA of the solver schedule in use (0: none fits)."""
        return _lib.tmr_schedule(self.h)

    def close(self):
        self.h.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def preprocess(frames: torch.Tensor, H: int | None = None, W: int | None = None, offset: int = 0,
               energy_frac: float = 0.999, stream: torch.cuda.Stream | None = None) -> dict:
    """Camera frames [K, H, W] (CUDA uint16, int16 holding uint16 bits, or float32)
    -> dict(y [M, K] float32, mask [M] uint8, energy [M] float64, n_inside [1] int32),
    the half-sampled, fiber-masked rows of Sec. 2.2 (tmr_preprocess).  y viewed as
    [M, J, N] is the input of Retriever.retrieve."""
    if not isinstance(frames, torch.Tensor) or not frames.is_cuda:
        raise TypeError("frames: a CUDA tensor is expected")
    if frames.dim() != 3:
        raise ValueError("frames: shape [K, H, W] expected")
    K, H, W = frames.shape
    ny, nx = _lib.half_grid(H, W, offset)
    M = ny * nx
    dev = frames.device
    out = dict(y=torch.empty((M, K), dtype=torch.float32, device=dev),
               mask=torch.empty((M,), dtype=torch.uint8, device=dev),
               energy=torch.empty((M,), dtype=torch.float64, device=dev),
               n_inside=torch.empty((1,), dtype=torch.int32, device=dev))
    wb = _lib.tmr_preprocess_workspace_bytes(K, H, W, offset)
    ws = torch.empty((max(wb, 1),), dtype=torch.uint8, device=dev)
    _lib.tmr_preprocess(frames.contiguous(), K, H, W, offset, energy_frac, out["y"], out["mask"],
                        out["energy"], out["n_inside"], ws, wb,
                        stream=stream.cuda_stream if stream is not None else None)
    out["workspace"] = ws  # kept alive until the asynchronous call has run
    return out
