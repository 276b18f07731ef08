"""Host-side check of the tensor-memory budget of the one-CTA-per-row solver.

The row solver keeps its L-BFGS pairs, and the Lanczos vectors of the spectral
start where they fit, in the SM's tensor memory: 128 lanes x 512 columns of
32-bit cells, each thread using columns of its own lane.  The column counts
come from host/device functions in solver_row.cuh; this test compiles a small
host program against that header (nvcc, no GPU needed) and checks, for every
row variant, option and Lanczos length, that the allocation is a power of two
within the SM's 512 columns and large enough for every value a CTA stores.
"""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2302_13524_gb300", "csrc")
INCLUDE = os.path.join(ROOT, "include")

PROGRAM = r"""
#include <cstdio>
#include "solver_row.cuh"
int main()
{
    using namespace tmr;
    const int Ns[3] = {512, 1024, 2048};
    for (int a = 0; a < 3; a++) {
        const int N = Ns[a];
        for (int J = 1; J <= kMaxMasks; J++) {
            if (!row_variant_fits(N, J)) continue;
            for (int m = 1; m <= kMaxMem; m++)
                for (int k = 0; k <= kMaxLanczos; k++) {
                    const int klz = row_tmem_klz(N, J, k > 0, k);
                    std::printf("%d %d %d %d %d %d %d %d %d %d\n", N, J, m, k, row_ept(N, J), row_quarter_warps(N, J),
                                row_tmem_block(N, J, m), row_tmem_lanczos_block(N, J, k > 0 ? k : 1), klz,
                                row_tmem_cols(N, J, m, klz));
                }
        }
    }
    return 0;
}
"""


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


@pytest.fixture(scope="module")
def table():
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "budget.cu")
        exe = os.path.join(d, "budget")
        with open(src, "w") as f:
            f.write(PROGRAM)
        r = subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I", INCLUDE,
                            "-I", CSRC, src, "-o", exe], capture_output=True, text=True)
        assert r.returncode == 0, r.stdout + r.stderr
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    rows = [tuple(int(x) for x in line.split()) for line in out.splitlines() if line.strip()]
    assert rows
    return rows


def test_every_variant_fits_the_sm(table):
    for N, J, m, k, ept, qw, pblock, lblock, klz, cols in table:
        BT = J * N // 16
        NW = BT // 32
        assert BT % 32 == 0 and BT <= 512
        # every element has exactly one owner: i = tid + e BT, e < ept
        assert ept * BT >= N and (ept - 1) * BT < N
        # warps w and w + 4 share lane quarter w mod 4: at most ceil(NW / 4) per quarter
        assert qw == -(-NW // 4)
        # a power of two of at least 32 columns, within the SM's 512
        assert 32 <= cols <= 512 and cols & (cols - 1) == 0, (N, J, m, k, cols)
        # the pairs: each thread's lane holds its ept elements of the m + 1
        # slots (s and y, re and im), and the quarter's warps' blocks fit
        assert pblock >= ept * (m + 1) * 4
        assert qw * pblock <= cols
        assert 128 * cols >= 2 * (m + 1) * N * 2
        assert qw * pblock <= 504  # the figure the header states for m <= 6


def test_lanczos_vectors_go_to_tensor_memory_exactly_where_they_fit(table):
    for N, J, m, k, ept, qw, pblock, lblock, klz, cols in table:
        if k == 0:
            assert klz == 0
            continue
        fits = qw * lblock <= 512
        assert klz == (k if fits else 0), (N, J, m, k)
        if klz:
            assert lblock >= 2 * ept * k and lblock % 8 == 0  # four vectors per 8-column load
            assert qw * lblock <= cols
            assert 128 * cols >= k * N * 2


def test_the_paper_scale_variant_uses_all_columns(table):
    by_key = {(r[0], r[1], r[2], r[3]): r for r in table}
    N, J, m, k, ept, qw, pblock, lblock, klz, cols = by_key[(2048, 4, 5, 16)]
    assert (ept, qw, klz, cols) == (4, 4, 16, 512)
    assert qw * pblock == 384 and qw * lblock == 512
    # J = 3 at N = 2048 has 12 warps and 6 elements per thread: its 16 Lanczos
    # vectors (576 columns) stay in global memory
    assert by_key[(2048, 3, 5, 16)][8] == 0
