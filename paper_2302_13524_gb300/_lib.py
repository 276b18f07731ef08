"""ctypes binding of libtmr (include/tmr.h): argument marshalling only.

Every function takes the same arguments as its C counterpart; arrays may be
torch tensors (CUDA or CPU) or numpy arrays, passed by their data pointers
after dtype/contiguity/size checks.  Errors raise TMRError.  There is no
fallback: if libtmr.so is missing or cannot be loaded, importing fails.
"""
from __future__ import annotations

import ctypes
import os
import re

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtmr.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "tmr.h")

TMR_OK, TMR_ERR_INVALID_ARG, TMR_ERR_UNSUPPORTED, TMR_ERR_OOM = 0, 1, 2, 3
TMR_ERR_CUDA, TMR_ERR_TIMEOUT, TMR_ERR_NUMERIC = 4, 5, 6
TMR_INIT_RANDOM, TMR_INIT_BP, TMR_INIT_SPECTRAL, TMR_INIT_LEARNED = 0, 1, 2, 3
TMR_ROW_MAXITER, TMR_ROW_CONVERGED, TMR_ROW_ZERO, TMR_ROW_NUMERIC = 0, 1, 2, 3
TMR_PREC_FP32 = 0
TMR_PREC_MIXED = 1
TMR_COST_INTENSITY, TMR_COST_AMPLITUDE = 0, 1
TMR_PIX_U16, TMR_PIX_F32 = 0, 1
TMR_LOSS_MSE, TMR_LOSS_PHASE = 0, 1
INIT = {"random": TMR_INIT_RANDOM, "bp": TMR_INIT_BP, "spectral": TMR_INIT_SPECTRAL,
        "learned": TMR_INIT_LEARNED}
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED", 3: "OOM", 4: "CUDA", 5: "TIMEOUT",
                6: "NUMERIC"}


class TMRError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class tmr_options(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("init", ctypes.c_int), ("seed", ctypes.c_ulonglong),
                ("power_iters", ctypes.c_int), ("clip", ctypes.c_double), ("tol", ctypes.c_double),
                ("phase_iters", ctypes.c_int), ("precision", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("workspace_limit", ctypes.c_size_t),
                ("schedule", ctypes.c_int), ("tune_cache", ctypes.c_char_p),
                ("wait_spins", ctypes.c_longlong), ("withhold_release", ctypes.c_int),
                ("probe_n1", ctypes.c_int), ("lanczos", ctypes.c_int), ("cost", ctypes.c_int),
                ("phase_tol", ctypes.c_double), ("dense", ctypes.c_int)]


class tmr_defocus_op(ctypes.Structure):
    _fields_ = [("ny", ctypes.c_int), ("nx", ctypes.c_int), ("H", ctypes.c_void_p),
                ("coef", ctypes.c_double), ("n_defocus", ctypes.c_int), ("kind", ctypes.c_int),
                ("wavelength", ctypes.c_double), ("na", ctypes.c_double), ("z_d", ctypes.c_double),
                ("pixel", ctypes.c_double), ("incident", ctypes.c_void_p)]


DEFOCUS_SAME_GRID, DEFOCUS_ANGULAR_2X = 0, 1


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libtmr.so not built ({LIB_PATH}); run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, ip, fp, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p
    H = ctypes.c_void_p
    sigs = {
        "tmr_default_options": ([ctypes.POINTER(tmr_options)], None),
        "tmr_create": ([ctypes.POINTER(H), ip, ip, ip, vp, ctypes.POINTER(tmr_defocus_op),
                        ctypes.POINTER(tmr_options), vp], ctypes.c_int),
        "tmr_forward": ([H, vp, fp], ctypes.c_int),
        "tmr_grad": ([H, vp, fp, fp, vp], ctypes.c_int),
        "tmr_retrieve": ([H, fp, fp, ip, vp, vp, vp, fp], ctypes.c_int),
        "tmr_retrieve_from": ([H, vp, fp, fp, ip, vp, vp, vp, fp], ctypes.c_int),
        "tmr_defocus_forward": ([H, vp, fp], ctypes.c_int),
        "tmr_defocus_fit": ([H, vp, fp, dp, vp], ctypes.c_int),
        "tmr_sync": ([H, ctypes.c_double], ctypes.c_int),
        "tmr_phase_fit_report": ([H, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "tmr_last_error": ([], ctypes.c_char_p),
        "tmr_workspace_bytes": ([H], ctypes.c_size_t),
        "tmr_schedule": ([H], ctypes.c_int),
        "tmr_mlp_create": ([ctypes.POINTER(vp), ip, ip, ip, ip, ctypes.c_ulonglong, vp], ctypes.c_int),
        "tmr_mlp_num_params": ([vp], ctypes.c_size_t),
        "tmr_mlp_set_params": ([vp, fp], ctypes.c_int),
        "tmr_mlp_get_params": ([vp, fp], ctypes.c_int),
        "tmr_mlp_forward": ([vp, fp, ip, fp], ctypes.c_int),
        "tmr_mlp_grad": ([vp, fp, fp, ip, fp, fp], ctypes.c_int),
        "tmr_mlp_train_step": ([vp, fp, fp, ip, ctypes.c_float, fp], ctypes.c_int),
        "tmr_mlp_destroy": ([vp], None),
        "tmr_mlp_set_loss": ([vp, ip], ctypes.c_int),
        "tmr_gemm_bf16": ([ip, ip, ip, vp, ip, vp, ip, fp, ip, vp], ctypes.c_int),
        "tmr_autotune_report": ([H, vp, vp, ip], ctypes.c_int),
        "tmr_set_init_model": ([H, vp], ctypes.c_int),
        "tmr_learned_rows": ([H], ctypes.c_longlong),
        "tmr_destroy": ([H], None),
        "tmr_retrieve_rows_static": ([ip, ip, ip, vp, fp, ip, ctypes.POINTER(tmr_options), vp, vp,
                                      vp, fp, vp], ctypes.c_int),
        "tmr_preprocess_workspace_bytes": ([ip, ip, ip, ip], ctypes.c_size_t),
        "tmr_preprocess": ([vp, ip, ip, ip, ip, ip, ctypes.c_double, fp, vp, dp, vp, vp, ctypes.c_size_t,
                            vp], ctypes.c_int),
        "tmr_half_sample": ([vp, ip, ip, ip, ip, ip, fp, vp], ctypes.c_int),
    }
    for name, (args, res) in sigs.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    return L


lib = _load()


def header_symbols(path: str = HEADER):
    """Function names declared in include/tmr.h."""
    with open(path) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(tmr_\w+)\s*\(", text, re.M)))


def _check(st: int):
    if st != TMR_OK:
        raise TMRError(st, lib.tmr_last_error().decode())


def _ptr(x, dtype=None, count=None, name="array"):
    """Data pointer of a torch tensor / numpy array (None -> NULL), with checks."""
    if x is None:
        return None
    mod = type(x).__module__
    if mod.startswith("torch"):
        import torch
        if dtype is not None:
            want = {"c64": torch.complex64, "f32": torch.float32, "i32": torch.int32,
                    "f64": torch.float64, "u8": torch.uint8}[dtype]
            if x.dtype != want:
                raise TypeError(f"{name}: dtype {x.dtype}, expected {want}")
        if not x.is_contiguous():
            raise ValueError(f"{name}: not contiguous")
        if count is not None and x.numel() != count:
            raise ValueError(f"{name}: {x.numel()} elements, expected {count}")
        return ctypes.c_void_p(x.data_ptr())
    import numpy as np
    if isinstance(x, np.ndarray):
        if dtype is not None:
            want = {"c64": np.complex64, "f32": np.float32, "i32": np.int32, "f64": np.float64,
                    "u8": np.uint8}[dtype]
            if x.dtype != want:
                raise TypeError(f"{name}: dtype {x.dtype}, expected {want}")
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{name}: not contiguous")
        if count is not None and x.size != count:
            raise ValueError(f"{name}: {x.size} elements, expected {count}")
        return ctypes.c_void_p(x.ctypes.data)
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    raise TypeError(f"{name}: unsupported array type {type(x)}")


def tmr_default_options(**overrides) -> tmr_options:
    o = tmr_options()
    lib.tmr_default_options(ctypes.byref(o))
    names = {f for f, _ in tmr_options._fields_}
    for k, v in overrides.items():
        if k not in names:  # ctypes would keep a misspelled option as a plain attribute
            raise TypeError(f"unknown option {k!r}")
        if k == "init" and isinstance(v, str):
            v = INIT[v]
        if k == "cost" and isinstance(v, str):
            v = {"intensity": TMR_COST_INTENSITY, "amplitude": TMR_COST_AMPLITUDE}[v]
        if k == "precision" and isinstance(v, str):
            v = {"fp32": TMR_PREC_FP32, "mixed": TMR_PREC_MIXED}[v]
        if k == "tune_cache" and isinstance(v, str):
            v = v.encode()
        setattr(o, k, v)
    return o


class Handle:
    """Owns a tmr_handle; sizes are kept for argument checks."""

    def __init__(self, raw, N, M, J, n_defocus, defocus_kind=DEFOCUS_SAME_GRID):
        self.raw = raw
        self.N, self.M, self.J, self.n_defocus = N, M, J, n_defocus
        self.defocus_kind = defocus_kind
        # pixels of one defocus image: the grid (kind 0) or the 2ny x 2nx grid (kind 1)
        self.defocus_pixels = M * (4 if defocus_kind == DEFOCUS_ANGULAR_2X else 1)
        self._keep = []

    def close(self):
        if self.raw:
            lib.tmr_destroy(self.raw)
            self.raw = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def tmr_create(N, M, J, masks, defocus_op=None, opt=None, stream=None) -> Handle:
    """defocus_op: None, dict(ny, nx, n_defocus, coef=0.05, H=None) (the same-grid
    operator), or dict(kind=1, ny, nx, n_defocus, wavelength, na, z_d, pixel,
    incident [n_defocus, N] complex64, H=None) (angular spectrum, 2x padding)."""
    dop = None
    keep = []
    if defocus_op is not None:
        kind = int(defocus_op.get("kind", DEFOCUS_SAME_GRID))
        nd = int(defocus_op["n_defocus"])
        Hp = _ptr(defocus_op.get("H"), "c64", M, "H")
        Ip = _ptr(defocus_op.get("incident"), "c64", nd * N, "incident")
        dop = tmr_defocus_op(int(defocus_op["ny"]), int(defocus_op["nx"]),
                             Hp.value if Hp is not None else None,
                             float(defocus_op.get("coef", 0.05)), nd, kind,
                             float(defocus_op.get("wavelength", 0.0)), float(defocus_op.get("na", 0.0)),
                             float(defocus_op.get("z_d", 0.0)), float(defocus_op.get("pixel", 0.0)),
                             Ip.value if Ip is not None else None)
        keep.append(defocus_op.get("H"))
        keep.append(defocus_op.get("incident"))
    if opt is None:
        opt = tmr_default_options()
    elif isinstance(opt, dict):
        opt = tmr_default_options(**opt)
    raw = ctypes.c_void_p()
    st = lib.tmr_create(ctypes.byref(raw), int(N), int(M), int(J), _ptr(masks, "c64", J * N, "masks"),
                        ctypes.byref(dop) if dop is not None else None, ctypes.byref(opt),
                        ctypes.c_void_p(stream) if stream else None)
    _check(st)
    return Handle(raw, N, M, J, dop.n_defocus if dop is not None else 0,
                  dop.kind if dop is not None else DEFOCUS_SAME_GRID)


def tmr_forward(h: Handle, T, Y):
    _check(lib.tmr_forward(h.raw, _ptr(T, "c64", h.M * h.N, "T"), _ptr(Y, "f32", h.M * h.J * h.N, "Y")))


def tmr_grad(h: Handle, T, Y, loss=None, G=None):
    _check(lib.tmr_grad(h.raw, _ptr(T, "c64", h.M * h.N, "T"), _ptr(Y, "f32", h.M * h.J * h.N, "Y"),
                        _ptr(loss, "f32", h.M, "loss"), _ptr(G, "c64", h.M * h.N, "G")))


def tmr_retrieve(h: Handle, y, y_def, iters, T_out, row_status=None, row_iters=None,
                 row_loss=None):
    _check(lib.tmr_retrieve(h.raw, _ptr(y, "f32", h.M * h.J * h.N, "y"),
                            _ptr(y_def, "f32", h.n_defocus * h.defocus_pixels, "y_def"), int(iters),
                            _ptr(T_out, "c64", h.M * h.N, "T_out"),
                            _ptr(row_status, "i32", h.M, "row_status"),
                            _ptr(row_iters, "i32", h.M, "row_iters"),
                            _ptr(row_loss, "f32", h.M, "row_loss")))


def tmr_retrieve_from(h: Handle, T_init, y, y_def, iters, T_out, row_status=None, row_iters=None,
                      row_loss=None):
    _check(lib.tmr_retrieve_from(h.raw, _ptr(T_init, "c64", h.M * h.N, "T_init"),
                                 _ptr(y, "f32", h.M * h.J * h.N, "y"),
                                 _ptr(y_def, "f32", h.n_defocus * h.defocus_pixels, "y_def"), int(iters),
                                 _ptr(T_out, "c64", h.M * h.N, "T_out"),
                                 _ptr(row_status, "i32", h.M, "row_status"),
                                 _ptr(row_iters, "i32", h.M, "row_iters"),
                                 _ptr(row_loss, "f32", h.M, "row_loss")))


def tmr_defocus_forward(h: Handle, T, Y_def):
    _check(lib.tmr_defocus_forward(h.raw, _ptr(T, "c64", h.M * h.N, "T"),
                                   _ptr(Y_def, "f32", h.n_defocus * h.defocus_pixels, "Y_def")))


def tmr_defocus_fit(h: Handle, T_est, y_def, phi=None, T_out=None):
    _check(lib.tmr_defocus_fit(h.raw, _ptr(T_est, "c64", h.M * h.N, "T_est"),
                               _ptr(y_def, "f32", h.n_defocus * h.defocus_pixels, "y_def"),
                               _ptr(phi, "f64", h.M, "phi"), _ptr(T_out, "c64", h.M * h.N, "T_out")))


def tmr_sync(h: Handle, timeout_s: float = 0.0):
    _check(lib.tmr_sync(h.raw, float(timeout_s)))


def tmr_last_error() -> str:
    return lib.tmr_last_error().decode()


def tmr_workspace_bytes(h: Handle) -> int:
    return int(lib.tmr_workspace_bytes(h.raw))


def tmr_autotune_report(h: Handle) -> dict:
    """{schedule code: mean ms of its timed runs} for the schedules the
    autotuner timed when the handle was made ({} when none were timed)."""
    codes = (ctypes.c_int * 8)()
    ms = (ctypes.c_float * 8)()
    n = lib.tmr_autotune_report(h.raw, codes, ms, 8)
    return {int(codes[i]): float(ms[i]) for i in range(min(n, 8))}


def tmr_phase_fit_report(h: Handle):
    """(loss g(phi), accepted iterations) of the last phase-offset fit."""
    loss, its = ctypes.c_double(), ctypes.c_int()
    _check(lib.tmr_phase_fit_report(h.raw, ctypes.byref(loss), ctypes.byref(its)))
    return loss.value, its.value


def tmr_schedule(h: Handle) -> int:
    return int(lib.tmr_schedule(h.raw))


def tmr_destroy(h: Handle):
    h.close()


class MLP:
    """Owns a tmr_mlp (the learned initialiser's network)."""

    def __init__(self, raw, dims):
        self.raw = raw
        self.dims = dims
        self.n_params = int(lib.tmr_mlp_num_params(raw))

    def close(self):
        if self.raw:
            lib.tmr_mlp_destroy(self.raw)
            self.raw = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def tmr_mlp_create(n_in, n_h1, n_h2, n_out, seed=0, stream=None) -> MLP:
    raw = ctypes.c_void_p()
    _check(lib.tmr_mlp_create(ctypes.byref(raw), int(n_in), int(n_h1), int(n_h2), int(n_out),
                              int(seed), ctypes.c_void_p(stream) if stream else None))
    return MLP(raw, (n_in, n_h1, n_h2, n_out))


def tmr_mlp_set_params(m: MLP, params):
    _check(lib.tmr_mlp_set_params(m.raw, _ptr(params, "f32", m.n_params, "params")))


def tmr_mlp_get_params(m: MLP, params):
    _check(lib.tmr_mlp_get_params(m.raw, _ptr(params, "f32", m.n_params, "params")))


def tmr_mlp_forward(m: MLP, X, B, Y):
    _check(lib.tmr_mlp_forward(m.raw, _ptr(X, "f32", B * m.dims[0], "X"), int(B),
                               _ptr(Y, "f32", B * m.dims[3], "Y")))


def tmr_mlp_grad(m: MLP, X, T, B, loss=None, grad=None):
    _check(lib.tmr_mlp_grad(m.raw, _ptr(X, "f32", B * m.dims[0], "X"), _ptr(T, "f32", B * m.dims[3], "T"),
                            int(B), _ptr(loss, "f32", 1, "loss"), _ptr(grad, "f32", m.n_params, "grad")))


def tmr_mlp_train_step(m: MLP, X, T, B, lr, loss=None):
    _check(lib.tmr_mlp_train_step(m.raw, _ptr(X, "f32", B * m.dims[0], "X"),
                                  _ptr(T, "f32", B * m.dims[3], "T"), int(B), float(lr),
                                  _ptr(loss, "f32", 1, "loss")))


def tmr_mlp_set_loss(m: MLP, kind):
    """TMR_LOSS_MSE or TMR_LOSS_PHASE (also "mse" / "phase")."""
    if isinstance(kind, str):
        kind = {"mse": TMR_LOSS_MSE, "phase": TMR_LOSS_PHASE}[kind]
    _check(lib.tmr_mlp_set_loss(m.raw, int(kind)))


def tmr_gemm_bf16(A, B, C, stream=None):
    """C = A B^T on the tensor cores; A [M][K], B [N][K] BF16 torch tensors (rows
    contiguous), C float32 [M][N]."""
    import torch
    for name, x, dt in (("A", A, torch.bfloat16), ("B", B, torch.bfloat16), ("C", C, torch.float32)):
        if x.dtype != dt or x.dim() != 2 or x.stride(1) != 1:
            raise TypeError(f"{name}: expected a 2-D {dt} tensor with contiguous rows")
    M, K = A.shape
    N = B.shape[0]
    if B.shape[1] != K or tuple(C.shape) != (M, N):
        raise ValueError("shapes: A [M][K], B [N][K], C [M][N]")
    _check(lib.tmr_gemm_bf16(M, N, K, ctypes.c_void_p(A.data_ptr()), A.stride(0), ctypes.c_void_p(B.data_ptr()),
                             B.stride(0), ctypes.c_void_p(C.data_ptr()), C.stride(0),
                             ctypes.c_void_p(stream) if stream else None))


def tmr_mlp_destroy(m: MLP):
    m.close()


def tmr_set_init_model(h: Handle, m):
    _check(lib.tmr_set_init_model(h.raw, m.raw if m is not None else None))


def tmr_learned_rows(h: Handle) -> int:
    return int(lib.tmr_learned_rows(h.raw))


def tmr_retrieve_rows_static(N, M, J, masks, y, iters, opt, T_out, row_status=None,
                             row_iters=None, row_loss=None, stream=None):
    """Allocation-free per-row retrieval (device arrays only, no handle)."""
    if opt is None:
        opt = tmr_default_options()
    elif isinstance(opt, dict):
        opt = tmr_default_options(**opt)
    _check(lib.tmr_retrieve_rows_static(
        int(N), int(M), int(J), _ptr(masks, "c64", J * N, "masks"),
        _ptr(y, "f32", M * J * N, "y"), int(iters), ctypes.byref(opt),
        _ptr(T_out, "c64", M * N, "T_out"), _ptr(row_status, "i32", M, "row_status"),
        _ptr(row_iters, "i32", M, "row_iters"), _ptr(row_loss, "f32", M, "row_loss"),
        ctypes.c_void_p(stream) if stream else None))


# ---- camera preprocessing ----------------------------------------------------
def half_grid(H: int, W: int, offset: int = 0) -> tuple[int, int]:
    """(ny, nx) of the half-sampled grid of an H x W frame."""
    return (int(H) - offset + 1) // 2, (int(W) - offset + 1) // 2


def _frames(frames, count):
    """(pointer, pixel type) of a frame stack: uint16 (or int16 holding the same
    bits) -> TMR_PIX_U16, float32 -> TMR_PIX_F32."""
    mod = type(frames).__module__
    if mod.startswith("torch"):
        import torch
        names = {torch.int16: TMR_PIX_U16, torch.float32: TMR_PIX_F32}
        if hasattr(torch, "uint16"):
            names[torch.uint16] = TMR_PIX_U16
        kind = names.get(frames.dtype)
        ok_contig = frames.is_contiguous()
        n = frames.numel()
        ptr = frames.data_ptr()
    else:
        import numpy as np
        frames = np.asarray(frames)
        kind = {np.dtype(np.uint16): TMR_PIX_U16, np.dtype(np.int16): TMR_PIX_U16,
                np.dtype(np.float32): TMR_PIX_F32}.get(frames.dtype)
        ok_contig = frames.flags["C_CONTIGUOUS"]
        n = frames.size
        ptr = frames.ctypes.data
    if kind is None:
        raise TypeError(f"frames: dtype {frames.dtype}, expected uint16 (or int16 bits) or float32")
    if not ok_contig:
        raise ValueError("frames: not contiguous")
    if n != count:
        raise ValueError(f"frames: {n} elements, expected {count}")
    return ctypes.c_void_p(ptr), kind


def tmr_preprocess_workspace_bytes(K: int, H: int, W: int, offset: int = 0) -> int:
    return int(lib.tmr_preprocess_workspace_bytes(int(K), int(H), int(W), int(offset)))


def tmr_preprocess(frames, K, H, W, offset, energy_frac, y, mask=None, energy=None, n_inside=None,
                   workspace=None, workspace_bytes=0, stream=None):
    """Camera frames [K][H][W] -> rows y [M][K], fiber mask, energies, count (device arrays)."""
    ny, nx = half_grid(H, W, offset)
    M = max(ny, 0) * max(nx, 0)
    fp_, kind = _frames(frames, int(K) * int(H) * int(W))
    _check(lib.tmr_preprocess(
        fp_, kind, int(K), int(H), int(W), int(offset), float(energy_frac),
        _ptr(y, "f32", M * int(K), "y"), _ptr(mask, "u8", M, "mask"), _ptr(energy, "f64", M, "energy"),
        _ptr(n_inside, "i32", 1, "n_inside"), _ptr(workspace, None, None, "workspace"),
        int(workspace_bytes), ctypes.c_void_p(stream) if stream else None))


def tmr_half_sample(frames, n, H, W, offset, out, stream=None):
    """Half-sampled frames: out [n][M] float32 (device arrays)."""
    ny, nx = half_grid(H, W, offset)
    M = max(ny, 0) * max(nx, 0)
    fp_, kind = _frames(frames, int(n) * int(H) * int(W))
    _check(lib.tmr_half_sample(fp_, kind, int(n), int(H), int(W), int(offset),
                               _ptr(out, "f32", int(n) * M, "out"),
                               ctypes.c_void_p(stream) if stream else None))
