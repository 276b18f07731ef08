"""The learned initialiser through the C ABI: the network's forward pass and
gradient against the FP64 oracle network (BF16 products, FP32 accumulation),
training on the GPU, and the per-row selection inside tmr_retrieve."""
import numpy as np
import pytest

import oracle
from helpers import problem, to_dev, to_np
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2302_13524_gb300 as tmr  # noqa: E402


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("dims,B", [((8, 6, 6, 4), 5), ((70, 40, 33, 20), 37), ((256, 96, 64, 130), 64),
                                    ((512, 264, 200, 136), 296)])
def test_mlp_forward_and_gradient_match_oracle(dims, B):
    """The last shape runs every product on the tcgen05 tensor cores (sizes of
    at least 128 x 128 x 64 with rows a multiple of 8), with tails in every
    dimension; the others run the mma.sync tile kernel."""
    rng = np.random.default_rng(sum(dims))
    with tmr.tmr_mlp_create(*dims, seed=3) as m:
        theta = (rng.standard_normal(m.n_params) * 0.3).astype(np.float32)
        tmr.tmr_mlp_set_params(m, theta)
        X = rng.standard_normal((B, dims[0])).astype(np.float32)
        T = rng.standard_normal((B, dims[3])).astype(np.float32)
        Y = torch.empty((B, dims[3]), dtype=torch.float32, device="cuda")
        tmr.tmr_mlp_forward(m, to_dev(X), B, Y)
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        G = torch.empty(m.n_params, dtype=torch.float32, device="cuda")
        tmr.tmr_mlp_grad(m, to_dev(X), to_dev(T), B, loss, G)
        torch.cuda.synchronize()
    Yo, _ = omlp.forward(theta.astype(np.float64), dims, X.astype(np.float64))
    Lo, Go = omlp.loss_grad(theta.astype(np.float64), dims, X, T)
    # BF16 operands (8-bit mantissa) with FP32 accumulation
    assert _rel(to_np(Y), Yo) <= 2e-2
    assert abs(float(to_np(loss)[0]) - Lo) <= 2e-2 * Lo
    g = to_np(G)
    assert _rel(g, Go) <= 3e-2
    assert np.dot(g, Go) / (np.linalg.norm(g) * np.linalg.norm(Go)) >= 0.999


@pytest.mark.parametrize("dims,B", [((8, 6, 6, 4), 5), ((256, 96, 64, 130), 64)])
def test_mlp_phase_invariant_loss_matches_oracle(dims, B):
    """TMR_LOSS_PHASE against oracle.mlp.loss_grad_phase: the same targets give
    the same loss and gradient (BF16 products), and turning every target row
    by its own global phase changes neither the library's loss nor its
    gradient beyond BF16 rounding."""
    rng = np.random.default_rng(sum(dims) + 1)
    n = dims[3] // 2
    with tmr.tmr_mlp_create(*dims, seed=4) as m:
        theta = (rng.standard_normal(m.n_params) * 0.3).astype(np.float32)
        tmr.tmr_mlp_set_params(m, theta)
        tmr.tmr_mlp_set_loss(m, "phase")
        X = rng.standard_normal((B, dims[0])).astype(np.float32)
        T = rng.standard_normal((B, dims[3])).astype(np.float32)
        t = (T[:, :n] + 1j * T[:, n:]) * np.exp(1j * rng.uniform(0, 2 * np.pi, B))[:, None]
        T2 = np.concatenate([t.real, t.imag], 1).astype(np.float32)
        out = {}
        for key, TT in (("T", T), ("T2", T2)):
            loss = torch.empty(1, dtype=torch.float32, device="cuda")
            G = torch.empty(m.n_params, dtype=torch.float32, device="cuda")
            tmr.tmr_mlp_grad(m, to_dev(X), to_dev(TT), B, loss, G)
            torch.cuda.synchronize()
            out[key] = (float(to_np(loss)[0]), to_np(G))
        with pytest.raises(tmr.TMRError):
            tmr.tmr_mlp_set_loss(m, 7)
    Lo, Go = omlp.loss_grad_phase(theta.astype(np.float64), dims, X, T)
    L, g = out["T"]
    assert abs(L - Lo) <= 2e-2 * Lo
    assert _rel(g, Go) <= 3e-2
    assert np.dot(g, Go) / (np.linalg.norm(g) * np.linalg.norm(Go)) >= 0.999
    L2, g2 = out["T2"]
    assert abs(L2 - L) <= 1e-3 * L and _rel(g2, g) <= 1e-2


def test_mlp_train_step_is_adam_on_its_gradient():
    """tmr_mlp_train_step against the oracle's Adam (FP64) parameter by
    parameter over 5 steps: at each step the gradient the library computes
    (tmr_mlp_grad, the same kernels the train step runs, deterministic) is fed
    to oracle.mlp.adam_step with the oracle's own moments, and the library's
    updated FP32 parameters must match the oracle's to FP32 rounding of the
    update."""
    rng = np.random.default_rng(7)
    dims, B, lr = (24, 16, 12, 10), 9, 3e-3
    with tmr.tmr_mlp_create(*dims, seed=2) as m:
        n = m.n_params
        theta = np.empty(n, np.float32)
        tmr.tmr_mlp_get_params(m, theta)
        th_o = theta.astype(np.float64)
        mo, vo = np.zeros(n), np.zeros(n)
        G = torch.empty(n, dtype=torch.float32, device="cuda")
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        for t in range(1, 6):
            X = to_dev(rng.standard_normal((B, dims[0])).astype(np.float32))
            T = to_dev(rng.standard_normal((B, dims[3])).astype(np.float32))
            tmr.tmr_mlp_grad(m, X, T, B, loss, G)
            G2 = torch.empty_like(G)
            tmr.tmr_mlp_grad(m, X, T, B, loss, G2)
            torch.cuda.synchronize()
            g = to_np(G).astype(np.float64)
            np.testing.assert_array_equal(to_np(G2), to_np(G))  # deterministic
            tmr.tmr_mlp_train_step(m, X, T, B, lr, loss)
            tmr.tmr_mlp_get_params(m, theta)
            th_o, mo, vo = omlp.adam_step(th_o, g, mo, vo, t, lr=lr)
            err = np.abs(theta.astype(np.float64) - th_o)
            assert np.all(err <= 1e-6 * np.abs(th_o) + 1e-4 * lr), (t, float(err.max()))
            th_o = theta.astype(np.float64)  # continue from the library's FP32 parameters


def test_mlp_training_learns_a_smooth_target():
    rng = np.random.default_rng(0)
    dims, B = (64, 128, 128, 16), 128
    A = rng.standard_normal((dims[3], dims[0])) / np.sqrt(dims[0])
    with tmr.tmr_mlp_create(*dims, seed=1) as m:
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        first = None
        for step in range(300):
            X = rng.standard_normal((B, dims[0])).astype(np.float32)
            T = np.tanh(X @ A.T).astype(np.float32)
            tmr.tmr_mlp_train_step(m, to_dev(X), to_dev(T), B, 2e-3, loss)
            if step == 0:
                first = float(to_np(loss)[0])
        last = float(to_np(loss)[0])
    assert last < 0.1 * first


def test_learned_start_seeds_and_falls_back():
    """TMR_INIT_LEARNED with power iterations: the network's proposal seeds the
    power iteration.  A network whose proposals are all zero (zero weights)
    leaves every row on the Philox seed: the retrieve equals the plain
    spectral one bit for bit and no row counts as seeded.  A network with
    nonzero proposals seeds every row.  Without power iterations the solver
    keeps, per row, the proposal or the random start, whichever has the lower
    loss: rows that kept the random start equal the plain random-start run."""
    N, M, J, iters = 256, 24, 4, 20
    T, d, Y = problem(N, M, J, seed=8)

    def run(init, pits, model=None):
        To = torch.empty((M, N), dtype=torch.complex64, device="cuda")
        with tmr.tmr_create(N, M, J, to_dev(d), None, dict(init=init, power_iters=pits, schedule=1)) as h:
            if init == "learned":
                with pytest.raises(tmr.TMRError):
                    tmr.tmr_retrieve(h, to_dev(Y), None, iters, To)  # no network yet
                tmr.tmr_set_init_model(h, model)
            tmr.tmr_retrieve(h, to_dev(Y), None, iters, To)
            torch.cuda.synchronize()
            kept = tmr.tmr_learned_rows(h) if init == "learned" else None
        return to_np(To), kept

    with tmr.tmr_mlp_create(J * N, 64, 64, 2 * N, seed=5) as zero_net, \
            tmr.tmr_mlp_create(J * N, 64, 64, 2 * N, seed=5) as net:
        tmr.tmr_mlp_set_params(zero_net, np.zeros(zero_net.n_params, np.float32))
        plain, _ = run("spectral", 40)
        z, kept_z = run("learned", 40, zero_net)
        assert kept_z == 0
        np.testing.assert_array_equal(z, plain)
        seeded, kept_s = run("learned", 40, net)
        assert kept_s == M
        assert np.mean(np.any(seeded != plain, axis=1)) > 0.9
        assert np.mean(oracle.fidelity_rows(seeded, T)) > 0.9
        rnd, _ = run("random", 0)
        judged, kept_j = run("learned", 0, net)
        differ = np.any(judged != rnd, axis=1)
        assert 0 <= kept_j <= M and int(differ.sum()) == kept_j


def test_learned_gain_measured_on_held_out_fibers():
    """What the trained network gains, measured on held-out fibers of a small
    family (N = 256, J = 4, shared input basis of R = 140 modes, 512 rows per
    fiber; 60 training fibers, 2 held-out fibers): the network is trained by
    the library's kernels (phase-invariant loss) on rows the plain solver
    retrieved, then the plain spectral start and the learned start (the
    proposal seeding the same power iteration) run with the same budgets.
    The learned start must give a higher mean fidelity at every budget of
    the grid, reach mean fidelity 0.98 with fewer operator products (power
    plus L-BFGS iterations; each applies Q and Q^H once), and beat the
    random start when no power iteration runs."""
    from paper_2302_13524_gb300 import learned_init as li
    import synth
    N, M, J, R = 256, 512, 4, 140
    _, d = synth.mask_phases(J, N, seed=0)

    def tm_fn(f):
        return synth.tm_family(M, N, R, fiber_seed=f, basis_seed=0)

    X, Tt = li.build_dataset(tm_fn, list(range(1, 61)), N, M, J, d, 1e4, 60, 60)
    P, I = (0, 10, 20, 30, 40, 50, 60, 80), (10, 20, 30, 40)
    budgets = [(p, i) for p in P for i in I]
    with tmr.tmr_mlp_create(J * N, 256, 256, 2 * N, seed=0) as model:
        hist = li.train(model, X, Tt, 30, 128, 3e-4)
        res = li.evaluate(model, tm_fn, [101, 102], N, M, J, d, 1e4, budgets,
                          arms=(("random", "fp32"), ("spectral", "fp32"), ("learned", "fp32")))
    assert all(np.isfinite(hist)) and hist[-1] < hist[0] - 0.01, hist  # the loss falls
    mean = {(arm, p, i): res[f"{arm}+fp32/{p}/{i}"]["mean"] for arm in ("spectral", "learned")
            for p in P for i in I}
    for p in (10, 20, 30, 40):
        for i in I:
            print(f"P={p} I={i}: spectral {mean['spectral', p, i]:.4f} learned {mean['learned', p, i]:.4f}")
            assert mean["learned", p, i] > mean["spectral", p, i], (p, i)

    def products(arm, bar):
        ok = [p + i for p in P for i in I if mean[arm, p, i] >= bar]
        return min(ok) if ok else 10 ** 9

    sp, le = products("spectral", 0.98), products("learned", 0.98)
    print(f"operator products to mean fidelity 0.98: spectral {sp}, learned {le}")
    assert le < sp
    for i in I:
        assert mean["learned", 0, i] > res[f"random+fp32/0/{i}"]["mean"] + 0.03
