"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: finite
differences of the cost, closed forms, invariants the paper states (Eq. 3's
normalisation and row bound, the maximum perplexity n-1 of Eq. 2, the value 1
of Eq. 9 for a collapsed map), library routines (scipy distances, brentq root
finding, torch autograd / AdamW) and brute-force loops on tiny inputs.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1812_09869_gb300 import synth


def _rand_P(z, seed):
    X, _ = synth.gaussian_mixture(z, 5, 2, seed=seed)
    P, _, st = O.affinities(X, min(5.0, (z - 1) / 2))
    assert st == 0
    return P


# ---------------------------------------------------------------- distances

def test_sqdist_matches_scipy():
    from scipy.spatial.distance import cdist
    X, _ = synth.gaussian_mixture(37, 7, 3, seed=11)
    np.testing.assert_allclose(O.sqdist(X), cdist(X.astype(np.float64), X.astype(np.float64),
                                                  "sqeuclidean"), rtol=1e-12, atol=1e-10)


# ---------------------------------------------------------------- perplexity search (Eq. 1-2)

def _perplexity_bits(cond_row):
    p = cond_row[cond_row > 0]
    return 2.0 ** (-(p * np.log2(p)).sum())


@pytest.mark.parametrize("perp", [5.0, 30.0, 80.0])
def test_every_row_hits_the_target_perplexity(perp):
    X, _ = synth.gaussian_mixture(300, 10, 4, seed=5)
    P, beta, cond, st = O.affinities(X, perp, want_cond=True)
    assert st == 0
    for i in range(300):
        # perplexity re-evaluated independently as 2^H with H in bits (Eq. 2)
        assert abs(_perplexity_bits(cond[i]) - perp) <= 1e-5
        assert abs(cond[i].sum() - 1.0) < 1e-12 and cond[i, i] == 0.0
    assert np.all(beta > 0)


def test_beta_matches_brentq_on_independent_entropy():
    from scipy.optimize import brentq
    X, _ = synth.gaussian_mixture(120, 6, 3, seed=8)
    D = O.sqdist(X)
    perp = 12.0
    for i in (0, 17, 119):
        d = np.delete(D[i], i)

        def H_bits(b):
            e = np.exp(-b * (d - d.min()))
            p = e / e.sum()
            p = p[p > 0]
            return -(p * np.log2(p)).sum() - math.log2(perp)

        ref = brentq(H_bits, 1e-8, 1e3, xtol=1e-15, rtol=1e-14)
        st, b, H, _ = O.row_beta(D[i], i, perp)
        assert st == 0
        assert abs(b - ref) <= 1e-8 * ref


def test_two_level_row_closed_form():
    """k neighbours at distance a, m = n-1-k at distance b > a:
    p_near = 1 / (k + m e^{-beta (b - a)}); the entropy has a closed form and
    beta(perp) is its root, found here by brentq on that formula."""
    from scipy.optimize import brentq
    k, m, a, b = 4, 15, 1.0, 3.5
    row = np.array([0.0] + [a] * k + [b] * m)  # point 0 is the row itself
    for perp in (5.0, 9.0, 15.0):
        def H_nats(beta):
            r = math.exp(-beta * (b - a))
            S = k + m * r
            pn, pf = 1.0 / S, r / S
            return -(k * pn * math.log(pn) + m * pf * math.log(pf)) - math.log(perp)
        ref = brentq(H_nats, 1e-9, 50.0, xtol=1e-15)
        st, beta, H, _ = O.row_beta(row, 0, perp)
        assert st == 0 and abs(beta - ref) <= 1e-8 * ref
        assert abs(math.exp(H) - perp) < 1e-8


def test_equidistant_points_give_maximum_perplexity():
    """All distances equal: p_{j|i} = 1/(n-1) for any beta and the perplexity is
    its maximum n-1 (Eq. 2 and the text after it)."""
    z = 9
    X = np.eye(z)  # regular simplex: every pairwise squared distance is 2
    P, beta, cond, st = O.affinities(X, z - 1.0, want_cond=True)
    assert st == 0
    off = ~np.eye(z, dtype=bool)
    np.testing.assert_allclose(cond[off], 1.0 / (z - 1), rtol=0, atol=1e-15)
    np.testing.assert_allclose(P[off], 1.0 / (z * (z - 1)), rtol=1e-14)
    # a target above the maximum cannot be met and is reported
    _, _, _, st2 = O.affinities(X, z + 0.5, want_cond=True)
    assert st2 == z


# ---------------------------------------------------------------- joint P (Eq. 3)

def test_joint_P_is_symmetric_normalised_and_row_bounded():
    X, _ = synth.gaussian_mixture(250, 8, 5, seed=3)
    z = 250
    P, _, st = O.affinities(X, 20.0)
    assert st == 0
    assert np.abs(P - P.T).max() == 0.0
    assert abs(P.sum() - 1.0) <= 1e-12
    assert np.all(np.diag(P) == 0.0)
    # sum_j p_ij > 1/(2n) for every i (text after Eq. 3)
    assert np.all(P.sum(1) > 1.0 / (2 * z))


def test_two_point_chunk_closed_form():
    """z = 2: p_{2|1} = p_{1|2} = 1, so P_12 = P_21 = 1/2; Q is 1/2 as well, so
    KL = 0 and the gradient vanishes for every map."""
    X = np.array([[0.0, 1.0], [2.0, -1.0]])
    P, beta, st = O.affinities(X, 1.0)
    np.testing.assert_array_equal(P, [[0.0, 0.5], [0.5, 0.0]])
    Y = np.array([[0.3, -1.2], [4.0, 2.5]])
    g, Z = O.gradient(P, Y)
    assert np.abs(g).max() < 1e-15
    assert abs(O.kl(P, Y)) < 1e-15


# ---------------------------------------------------------------- gradient (Eq. 4-6)

def test_gradient_matches_central_differences_of_kl():
    z = 14
    P = _rand_P(z, 21)
    rng = np.random.default_rng(0)
    Y = rng.standard_normal((z, 2))
    g, _ = O.gradient(P, Y)
    h = 1e-6
    fd = np.zeros_like(Y)
    for i in range(z):
        for k in range(2):
            Yp, Ym = Y.copy(), Y.copy()
            Yp[i, k] += h
            Ym[i, k] -= h
            fd[i, k] = (O.kl(P, Yp) - O.kl(P, Ym)) / (2 * h)
    assert np.abs(g - fd).max() <= 1e-6 * np.abs(g).max()


def test_gradient_three_dimensional_map_matches_central_differences():
    z = 9
    P = _rand_P(z, 22)
    Y = np.random.default_rng(1).standard_normal((z, 3)) * 2.0
    g, _ = O.gradient(P, Y)
    h = 1e-6
    fd = np.zeros_like(Y)
    for i in range(z):
        for k in range(3):
            Yp, Ym = Y.copy(), Y.copy()
            Yp[i, k] += h
            Ym[i, k] -= h
            fd[i, k] = (O.kl(P, Yp) - O.kl(P, Ym)) / (2 * h)
    assert np.abs(g - fd).max() <= 1e-6 * np.abs(g).max()


def test_gradient_sums_to_zero_and_respects_rigid_motions():
    z = 60
    P = _rand_P(z, 23)
    rng = np.random.default_rng(2)
    Y = rng.standard_normal((z, 2)) * 3
    g, Z = O.gradient(P, Y)
    scale = np.abs(g).max()
    assert np.abs(g.sum(0)).max() <= 1e-13 * z * scale
    g2, Z2 = O.gradient(P, Y + np.array([7.5, -3.0]))
    assert np.abs(g2 - g).max() <= 1e-12 * scale and abs(Z2 - Z) <= 1e-12 * Z
    th = 0.7
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    g3, _ = O.gradient(P, Y @ R.T)
    assert np.abs(g3 - g @ R.T).max() <= 1e-12 * scale


def test_gradient_of_selected_rows_matches_central_differences():
    """The row-restricted form of Eq. 6 (for chunks whose P is too large to
    hold whole) against central differences of the KL at those rows, 2-D and
    3-D maps, rows in any order."""
    for od, z, seed in ((2, 12, 25), (3, 8, 26)):
        P = _rand_P(z, seed)
        Y = np.random.default_rng(seed).standard_normal((z, od)) * 1.5
        rows = np.array([z - 1, 0, 3])
        g = O.gradient_rows(P[rows], rows, Y, O.cauchy_Z(Y))
        h = 1e-6
        fd = np.zeros((len(rows), od))
        for r, i in enumerate(rows):
            for k in range(od):
                Yp, Ym = Y.copy(), Y.copy()
                Yp[i, k] += h
                Ym[i, k] -= h
                fd[r, k] = (O.kl(P, Yp) - O.kl(P, Ym)) / (2 * h)
        assert np.abs(g - fd).max() <= 1e-6 * np.abs(fd).max()


def test_Z_brute_force():
    Y = np.random.default_rng(3).standard_normal((7, 2))
    ref = sum(1.0 / (1.0 + ((Y[k] - Y[l]) ** 2).sum())
              for k in range(7) for l in range(7) if k != l)
    assert abs(O.cauchy_Z(Y) - ref) <= 1e-14 * ref


# ---------------------------------------------------------------- costs (Eq. 5, Eq. 9)

def test_kl_and_normalized_cost_brute_force():
    z = 6
    P = _rand_P(z, 24)
    Y = np.random.default_rng(4).standard_normal((z, 2))
    w = np.array([[0.0 if i == j else 1.0 / (1.0 + ((Y[i] - Y[j]) ** 2).sum())
                   for j in range(z)] for i in range(z)])
    Q = w / w.sum()
    kl = sum(P[i, j] * math.log(P[i, j] / Q[i, j]) for i in range(z) for j in range(z) if i != j)
    ce = -sum(P[i, j] * math.log(Q[i, j]) for i in range(z) for j in range(z) if i != j)
    assert abs(O.kl(P, Y) - kl) <= 1e-13
    assert abs(O.normalized_cost(P, Y) - ce / (math.log(z) + math.log(z - 1))) <= 1e-13


def test_normalized_cost_is_one_for_a_collapsed_map():
    """All y equal: q_ij = 1/(n(n-1)) (Eq. 7), so Eq. 9 equals 1 exactly."""
    z = 40
    P = _rand_P(z, 25)
    Y = np.tile([[0.25, -1.5]], (z, 1))
    assert abs(O.normalized_cost(P, Y) - 1.0) <= 1e-14


def test_normalized_cost_near_one_for_random_initial_map():
    """A random initial map (tiny N(0, 1e-4) spread) gives a value very close to
    1 (text after Eq. 9)."""
    X, _ = synth.gaussian_mixture(400, 10, 4, seed=9)
    P, _, _ = O.affinities(X, 30.0)
    Y = synth.init_gaussian(400, 2, 1e-4, seed=1).astype(np.float64)
    assert abs(O.normalized_cost(P, Y) - 1.0) < 1e-6


def test_embedding_size_is_bounding_box_diagonal():
    Y = np.array([[0.0, 0.0], [3.0, 1.0], [1.0, 4.0], [2.0, 2.0]])
    assert O.embedding_size(Y) == pytest.approx(5.0, abs=1e-15)  # box 3 x 4


# ---------------------------------------------------------------- update (Eq. 12, Eq. 13)

def test_update_without_momentum_or_gains_is_plain_descent():
    rng = np.random.default_rng(5)
    Y = rng.standard_normal((10, 2))
    g = rng.standard_normal((10, 2))
    vel = np.zeros((10, 2))
    gains = np.ones((10, 2))
    Y0 = Y.copy()
    O.update(Y, vel, gains, g, lr=0.3, momentum=0.0, use_gains=0)
    np.testing.assert_allclose(Y, Y0 - 0.3 * g, rtol=0, atol=1e-15)


def test_update_momentum_term_reproduces_previous_displacement():
    """Eq. 12: y(t) = y(t-1) - eta g + alpha (y(t-1) - y(t-2))."""
    rng = np.random.default_rng(6)
    Y = rng.standard_normal((5, 2))
    vel = np.zeros((5, 2))
    gains = np.ones((5, 2))
    g1, g2 = rng.standard_normal((5, 2)), rng.standard_normal((5, 2))
    O.update(Y, vel, gains, g1, lr=0.5, momentum=0.8, use_gains=0)
    Ym1 = Y.copy()
    Ym2 = Ym1 + 0.5 * g1
    O.update(Y, vel, gains, g2, lr=0.5, momentum=0.8, use_gains=0)
    np.testing.assert_allclose(Y, Ym1 - 0.5 * g2 + 0.8 * (Ym1 - Ym2), atol=1e-14)


def test_gains_grow_on_sign_change_decay_otherwise_with_floor():
    Y = np.zeros((1, 2))
    vel = np.array([[1.0, 1.0]])
    gains = np.ones((1, 2))
    # coordinate 0: grad > 0 with vel > 0 (agree) -> x0.8; coordinate 1: grad < 0 -> +0.2
    O.update(Y, vel, gains, np.array([[1.0, -1.0]]), lr=0.0, momentum=1.0)
    np.testing.assert_allclose(gains, [[0.8, 1.2]], atol=1e-15)
    for _ in range(60):
        O.update(Y, vel, gains, np.array([[1.0, -1.0]]), lr=0.0, momentum=1.0)
    assert gains[0, 0] == pytest.approx(0.01, abs=1e-15)


def test_descent_step_lowers_the_kl():
    """The sign reading of Eq. 12: a small step along -grad lowers Eq. 5."""
    z = 30
    P = _rand_P(z, 26)
    Y = np.random.default_rng(7).standard_normal((z, 2))
    g, _ = O.gradient(P, Y)
    Y2, vel, gains = Y.copy(), np.zeros_like(Y), np.ones_like(Y)
    O.update(Y2, vel, gains, g, lr=1e-2, momentum=0.0, use_gains=0)
    assert O.kl(P, Y2) < O.kl(P, Y)


def test_paper_learning_rate_eq13():
    Y = np.array([[-1.0, 0.5], [3.0, 0.0], [0.0, 2.0], [1.0, 1.0], [2.0, -0.5]])
    assert O.paper_lr(Y) == pytest.approx(math.log(4) * (3.0 - (-1.0)) / 2, rel=1e-15)


# ---------------------------------------------------------------- the ptSNE cycle

def test_single_chunk_run_equals_partial_tsne():
    X, _ = synth.gaussian_mixture(150, 6, 3, seed=12)
    perm = synth.permutations(150, 1, seed=1)
    off = np.array([0, 150])
    Y0 = synth.init_gaussian(150, 2, 1e-4, seed=2)
    prm = O.params(perplexity=10.0, iters=20, epochs=1)
    Y, cost = O.ptsne_run(X, Y0, perm, off, prm)
    Yc, kl, nc, st = O.partial_tsne(X[perm[0]], Y0[perm[0]], prm)
    np.testing.assert_array_equal(Y[perm[0]], Yc)
    assert cost[0, 0] == kl and cost[0, 1] == nc


def test_ptsne_cost_decreases_over_epochs():
    """As the mapping improves the (average, per-chunk) cost decreases (ptSNE
    section, cost and size monitoring)."""
    X, _ = synth.gaussian_mixture(1200, 8, 6, seed=13)
    off = synth.equal_chunk_offsets(1200, 4)
    perms = synth.permutations(1200, 4, seed=3)
    Y0 = synth.init_gaussian(1200, 2, 1e-4, seed=4)
    prm = O.params(perplexity=20.0, iters=40, epochs=4)
    Y, cost = O.ptsne_run(X, Y0, perms, off, prm)
    assert cost[-1, 1] < cost[0, 1] < 1.0
    assert O.embedding_size(Y) > O.embedding_size(Y0)


# ---------------------------------------------------------------- learned mapper oracle

def _mlp_weights(din, seed, h=16):
    rng = np.random.default_rng(seed)
    return {"W1": rng.standard_normal((h, din)) * 0.4, "b1": rng.standard_normal(h) * 0.1,
            "W2": rng.standard_normal((h, h)) * 0.3, "b2": rng.standard_normal(h) * 0.1,
            "W3": rng.standard_normal((2, h)) * 0.3, "b3": rng.standard_normal(2) * 0.1}


def test_mlp_gradient_matches_central_differences():
    W = _mlp_weights(5, 0)
    rng = np.random.default_rng(1)
    x, t = rng.standard_normal((7, 5)), rng.standard_normal((7, 2))
    L, g = O.mlp_loss_grad(W, x, t)
    h = 1e-6
    for k in W:
        flat = W[k].reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 11)):
            Wp = {kk: vv.copy() for kk, vv in W.items()}
            Wm = {kk: vv.copy() for kk, vv in W.items()}
            Wp[k].reshape(-1)[idx] += h
            Wm[k].reshape(-1)[idx] -= h
            fd = (O.mlp_loss_grad(Wp, x, t)[0] - O.mlp_loss_grad(Wm, x, t)[0]) / (2 * h)
            assert abs(fd - g[k].reshape(-1)[idx]) <= 1e-7 * max(1.0, abs(fd))


def test_mlp_matches_torch_autograd_fp64():
    torch = pytest.importorskip("torch")
    W = _mlp_weights(9, 2)
    rng = np.random.default_rng(3)
    x, t = rng.standard_normal((11, 9)), rng.standard_normal((11, 2))
    L, g = O.mlp_loss_grad(W, x, t)
    T = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in W.items()}
    xt, tt = torch.tensor(x), torch.tensor(t)
    h1 = torch.nn.functional.gelu(xt @ T["W1"].T + T["b1"])
    h2 = torch.nn.functional.gelu(h1 @ T["W2"].T + T["b2"])
    y = h2 @ T["W3"].T + T["b3"]
    Lt = 0.5 * ((y - tt) ** 2).sum() / x.shape[0]
    Lt.backward()
    assert abs(Lt.item() - L) <= 1e-13
    for k in W:
        np.testing.assert_allclose(g[k], T[k].grad.numpy(), rtol=1e-11, atol=1e-13)


def test_adamw_matches_torch():
    torch = pytest.importorskip("torch")
    W = _mlp_weights(4, 4)
    rng = np.random.default_rng(5)
    m = {k: np.zeros_like(v) for k, v in W.items()}
    v = {k: np.zeros_like(vv) for k, vv in W.items()}
    T = {k: torch.tensor(val.copy(), dtype=torch.float64, requires_grad=True) for k, val in W.items()}
    opt = torch.optim.AdamW([{"params": [T[k] for k in W if k.startswith("W")], "weight_decay": 1e-4},
                             {"params": [T[k] for k in W if k.startswith("b")], "weight_decay": 0.0}],
                            lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    for step in range(1, 4):
        g = {k: rng.standard_normal(val.shape) for k, val in W.items()}
        O.adamw_step(W, g, m, v, step)
        for k in W:
            T[k].grad = torch.tensor(g[k])
        opt.step()
    for k in W:
        np.testing.assert_allclose(W[k], T[k].detach().numpy(), rtol=1e-12, atol=1e-15)


def test_knn_preservation_brute_force():
    rng = np.random.default_rng(6)
    X = rng.standard_normal((40, 5))
    assert O.knn_preservation(X, X, X, X, k=5) == 1.0
    Y = rng.standard_normal((40, 2))
    # brute force: neighbour sets by explicit distance loops
    def nn(A, i, k):
        d = [(((A[i] - A[j]) ** 2).sum(), j) for j in range(len(A)) if j != i]
        return {j for _, j in sorted(d)[:k]}
    ref = np.mean([len(nn(X, i, 5) & nn(Y, i, 5)) / 5 for i in range(40)])
    assert O.knn_preservation(X, X, Y, Y, k=5) == pytest.approx(ref, abs=1e-15)


def test_affinities_from_distances_equal_point_affinities():
    """The point form is the distance form applied to squared distances."""
    X = np.random.default_rng(40).standard_normal((70, 6))
    P1, b1, _ = O.affinities(X, 12.0)
    P2, b2, bad = O.affinities_from_distances(O.sqdist(X), 12.0)
    assert bad == 0
    assert np.array_equal(P1, P2) and np.array_equal(b1, b2)


def test_affinities_from_graph_path_lengths():
    """Precomputed non-Euclidean dissimilarities (shortest-path lengths of a
    random connected graph): every row reaches the target perplexity (2^H
    re-evaluated here from beta and the row, and beta equal to an independent
    brentq root), P is symmetric with unit mass."""
    from scipy.optimize import brentq
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import shortest_path
    rng = np.random.default_rng(41)
    z, perp = 120, 15.0
    W = np.zeros((z, z))
    for i in range(z):                       # a ring keeps the graph connected, plus random chords
        W[i, (i + 1) % z] = rng.uniform(0.5, 2.0)
    for _ in range(3 * z):
        i, j = rng.integers(0, z, 2)
        if i != j:
            W[i, j] = rng.uniform(0.5, 4.0)
    G = shortest_path(csr_matrix(W), directed=False)
    P, beta, bad = O.affinities_from_distances(G, perp)
    assert bad == 0
    assert np.allclose(P, P.T, rtol=0, atol=0) and abs(P.sum() - 1.0) < 1e-12
    for i in range(z):
        d = np.delete(G[i], i)
        t = d - d.min()

        def H(b):
            e = np.exp(-b * t)
            p = e / e.sum()
            return -(p[p > 0] * np.log(p[p > 0])).sum()
        assert abs(np.exp(H(beta[i])) - perp) <= 1e-5
        if i % 20 == 0:
            root = brentq(lambda b: H(b) - np.log(perp), 1e-8, 1e3, xtol=1e-14, rtol=1e-14)
            assert abs(beta[i] - root) <= 1e-6 * root


def test_layers_one_is_the_plain_cycle():
    X = np.random.default_rng(42).standard_normal((150, 5))
    off = np.array([0, 50, 100, 150])
    perms = np.stack([np.random.default_rng(43 + e).permutation(150) for e in range(2)]).astype(np.int32)
    Y0 = np.random.default_rng(44).standard_normal((150, 2)) * 1e-2
    prm = O.params(perplexity=8.0, iters=10, epochs=2)
    Y1, c1 = O.ptsne_run(X, Y0, perms, off, prm)
    Y2, c2 = O.ptsne_run_layers(X, Y0, perms, off, 1, prm)
    assert np.array_equal(Y1, Y2) and np.array_equal(c1, c2)


def test_layers_chain_matches_an_explicit_assembly():
    """Thread t of a layered epoch is the partial t-SNE of elementary chunks
    t .. t+L-1 (mod T), slot k reading and writing layer k: restated here with
    explicit loops over threads and slots."""
    rng = np.random.default_rng(45)
    n, T, L = 120, 4, 3
    X = rng.standard_normal((n, 4))
    off = np.array([0, 30, 55, 90, 120])
    perm = rng.permutation(n).astype(np.int32)
    Y0 = rng.standard_normal((L * n, 2)) * 1e-2
    prm = O.params(perplexity=10.0, iters=8, epochs=1)
    Y, cost = O.ptsne_run_layers(X, Y0, perm[None, :], off, L, prm)
    Yref = Y0.copy()
    kls = []
    for t in range(T):
        rows = []
        for k in range(L):
            c = (t + k) % T
            rows += [(k, int(p)) for p in perm[off[c]:off[c + 1]]]
        Xc = np.array([X[p] for _, p in rows])
        Yc = np.array([Y0[k * n + p] for k, p in rows])
        Yt, kl, _, st = O.partial_tsne(Xc, Yc, prm)
        assert st == 0
        for q, (k, p) in enumerate(rows):
            Yref[k * n + p] = Yt[q]
        kls.append(kl)
    assert np.array_equal(Y, Yref)
    assert cost[0, 0] == pytest.approx(np.mean(kls), rel=1e-15)


def test_kde_cell_masses_match_gaussian_integrals():
    """For one kernel, S times the density at a cell centre approximates the
    exact Gaussian mass of the cell (products of erf differences) to second
    order in the cell size, and the masses sum to 1 over a grid covering
    +-8 standard deviations."""
    from scipy.special import erf
    beta, y = 3.0, np.array([[0.13, -0.21]])
    s = 1.0 / math.sqrt(2.0 * beta)                  # per-axis standard deviation
    box = (-8 * s + 0.13, 8 * s + 0.13, -8 * s - 0.21, 8 * s - 0.21)
    g = 400
    f = O.kde_grid(y, np.array([beta]), g, g, box)
    edges_x = np.linspace(box[0], box[1], g + 1)
    edges_y = np.linspace(box[2], box[3], g + 1)
    mx = 0.5 * np.diff(erf((edges_x - y[0, 0]) / (math.sqrt(2) * s)))
    my = 0.5 * np.diff(erf((edges_y - y[0, 1]) / (math.sqrt(2) * s)))
    exact = np.outer(my, mx)
    h = (box[1] - box[0]) / g
    assert np.abs(f - exact).max() <= 0.5 * (h / s) ** 2 * exact.max()
    assert abs(f.sum() - 1.0) <= 1e-6


def test_kde_is_the_average_of_the_kernels():
    """n points: the estimate is the mean of the one-point estimates (the
    S / n normalisation), and scales with beta as a 2-D density."""
    rng = np.random.default_rng(47)
    Y = rng.standard_normal((5, 2))
    beta = rng.uniform(0.5, 4.0, 5)
    box = (-4.0, 4.0, -3.0, 5.0)
    f = O.kde_grid(Y, beta, 60, 50, box)
    parts = [O.kde_grid(Y[j:j + 1], beta[j:j + 1], 60, 50, box) for j in range(5)]
    assert np.allclose(f, np.mean(parts, axis=0), rtol=1e-13, atol=0)
