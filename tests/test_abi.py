"""CPU checks of the C-ABI library: it loads, exports every function that
include/tmr.h declares, and its host-only entry points behave."""
import ctypes

import pytest


def test_library_exports_every_declared_symbol():
    tmr = pytest.importorskip("paper_2302_13524_gb300")
    names = tmr.header_symbols()
    assert len(names) >= 12
    raw = ctypes.CDLL(tmr.LIB_PATH)
    for n in names:
        assert hasattr(raw, n), n


def test_default_options_and_errors_without_device():
    tmr = pytest.importorskip("paper_2302_13524_gb300")
    o = tmr.tmr_default_options()
    assert (o.m, o.init, o.power_iters, o.phase_iters) == (5, tmr.TMR_INIT_SPECTRAL, 100, 100)
    assert o.clip == 2.0 and o.tol == 0.0
    o2 = tmr.tmr_default_options(init="bp", m=3)
    assert (o2.init, o2.m) == (tmr.TMR_INIT_BP, 3)
    import numpy as np
    with pytest.raises(tmr.TMRError):
        tmr.tmr_create(64, 4, 4, np.ones(4 * 64, np.complex64), opt=dict(m=0))
    with pytest.raises(TypeError):
        tmr.tmr_create(64, 4, 4, np.ones(4 * 64, np.complex128))
    tmr.lib.tmr_destroy(None)  # NULL is allowed


def test_header_documents_every_entry_point():
    tmr = pytest.importorskip("paper_2302_13524_gb300")
    text = open(tmr._lib.HEADER).read()
    for n in tmr.header_symbols():
        assert text.count(n) >= 1
    for sec in ("Eq. optTMsmall2", "Eq. derivative", "Eq. optphase", "Eq. phaseoffset"):
        assert sec in text


def test_preprocess_workspace_size():
    """Scratch of tmr_preprocess: one 64-bit energy partial per (256-frame chunk,
    pixel), one key per pixel, the mask and a flag, each block 256-byte aligned;
    0 for sizes without a half grid."""
    tmr = pytest.importorskip("paper_2302_13524_gb300")
    for K, H, W, off in [(8192, 256, 128, 0), (1, 3, 3, 1), (513, 9, 130, 1), (96, 37, 50, 0)]:
        ny, nx = tmr.half_grid(H, W, off)
        M, C = ny * nx, -(-K // 256)
        low = 8 * M * C + 8 * M + M + 4
        got = tmr.tmr_preprocess_workspace_bytes(K, H, W, off)
        assert low <= got <= low + 4 * 256, (K, H, W, off, got, low)
    for K, H, W, off in [(0, 8, 8, 0), (4, 0, 8, 0), (4, 8, 8, 2), (4, 1, 8, 1), (4, 8, 1, 1), (4, 8, 8, -1)]:
        assert tmr.tmr_preprocess_workspace_bytes(K, H, W, off) == 0


def test_preprocess_argument_errors_before_any_device_work():
    """Argument checks that precede every CUDA call return INVALID_ARG with a
    message, on a machine without a GPU too."""
    tmr = pytest.importorskip("paper_2302_13524_gb300")
    import ctypes as ct
    lib = tmr.lib
    dummy = ct.c_void_p(16)  # never dereferenced: each call fails its checks first
    cases = [
        (dummy, tmr.TMR_PIX_U16, 4, 8, 8, 2, 0.9, dummy, dummy, 1 << 20),   # offset
        (dummy, tmr.TMR_PIX_U16, 0, 8, 8, 0, 0.9, dummy, dummy, 1 << 20),   # K
        (dummy, tmr.TMR_PIX_U16, 4, 1, 8, 1, 0.9, dummy, dummy, 1 << 20),   # empty half grid
        (dummy, 7, 4, 8, 8, 0, 0.9, dummy, dummy, 1 << 20),                 # pixel type
        (dummy, tmr.TMR_PIX_F32, 4, 8, 8, 0, 0.0, dummy, dummy, 1 << 20),   # fraction
        (dummy, tmr.TMR_PIX_F32, 4, 8, 8, 0, 1.01, dummy, dummy, 1 << 20),  # fraction
        (dummy, tmr.TMR_PIX_F32, 4, 8, 8, 0, float("nan"), dummy, dummy, 1 << 20),
        (None, tmr.TMR_PIX_F32, 4, 8, 8, 0, 0.9, dummy, dummy, 1 << 20),    # NULL frames
        (dummy, tmr.TMR_PIX_F32, 4, 8, 8, 0, 0.9, None, dummy, 1 << 20),    # NULL y
        (dummy, tmr.TMR_PIX_F32, 4, 8, 8, 0, 0.9, dummy, None, 1 << 20),    # NULL workspace
        (dummy, tmr.TMR_PIX_F32, 4, 8, 8, 0, 0.9, dummy, dummy, 16),        # short workspace
        (dummy, tmr.TMR_PIX_U16, 65535 * 256 + 1, 8, 8, 0, 0.9, dummy, dummy, 1 << 40),  # K too large
    ]
    for fr, pt, K, H, W, off, frac, y, ws, wb in cases:
        st = lib.tmr_preprocess(fr, pt, K, H, W, off, frac, y, None, None, None, ws, wb, None)
        assert st == tmr.TMR_ERR_INVALID_ARG, (pt, K, H, W, off, frac)
        assert lib.tmr_last_error().decode().startswith("tmr_preprocess")
    for fr, pt, n, H, W, off, out in [(dummy, tmr.TMR_PIX_U16, 4, 8, 8, 3, dummy), (dummy, 9, 4, 8, 8, 0, dummy),
                                      (None, tmr.TMR_PIX_U16, 4, 8, 8, 0, dummy),
                                      (dummy, tmr.TMR_PIX_U16, 4, 8, 8, 0, None)]:
        assert lib.tmr_half_sample(fr, pt, n, H, W, off, out, None) == tmr.TMR_ERR_INVALID_ARG
    with pytest.raises(TypeError):
        import torch
        tmr.preprocess(torch.zeros((2, 4, 4), dtype=torch.int16))  # not on a GPU


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of tmr_options and tmr_defocus_op have the C
    compiler's field offsets and sizes (a field added to the header but not to
    the binding, or in another order, fails here)."""
    import shutil
    import subprocess
    tmr = pytest.importorskip("paper_2302_13524_gb300")
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    import os
    inc = os.path.dirname(tmr._lib.HEADER)
    lines = []
    for cname, cls in (("tmr_options", tmr._lib.tmr_options), ("tmr_defocus_op", tmr._lib.tmr_defocus_op)):
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    src = tmp_path / "layout.c"
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"tmr.h\"\nint main(void){\n"
                   + "\n".join(lines) + "\nreturn 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {(a, b): int(c) for a, b, c in (ln.split() for ln in out if ln)}
    for cname, cls in (("tmr_options", tmr._lib.tmr_options), ("tmr_defocus_op", tmr._lib.tmr_defocus_op)):
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)


def test_arrays_on_another_gpu_are_refused():
    """An array on a GPU other than the current one is refused with
    INVALID_ARG before any kernel could touch it (only where two GPUs are
    visible; one GPU or none: skipped)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available() or torch.cuda.device_count() < 2:
        pytest.skip("needs two visible GPUs")
    tmr = pytest.importorskip("paper_2302_13524_gb300")
    N, M, J = 64, 4, 4
    d = torch.ones((J, N), dtype=torch.complex64, device="cuda:0")
    with tmr.tmr_create(N, M, J, d) as h:
        T_other = torch.zeros((M, N), dtype=torch.complex64, device="cuda:1")
        Y = torch.empty((M, J, N), dtype=torch.float32, device="cuda:0")
        with pytest.raises(tmr.TMRError) as ei:
            tmr.tmr_forward(h, T_other, Y)
        assert ei.value.status == tmr.TMR_ERR_INVALID_ARG
