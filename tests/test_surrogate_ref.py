"""Pins of the surrogate's CPU reference (oracle/surrogate_ref.py) against
definitions it does not share: bf16 rounding on hand-worked values, the
convolution against numpy.correlate and brute-force loops, the bin assembly
against a brute-force sum and its gradient as its exact transpose, the
gradients against central differences of the forward pass, Adam's first step
against its closed form (a signed step of size lr)."""
import math

import numpy as np

from oracle import surrogate_ref as R


def test_bf16_rounding_hand_values():
    x = np.array([1.0, 1 + 2 ** -8, 1 + 2 ** -8 + 2 ** -20, 1 + 3 * 2 ** -8, -2.5, 0.0, 2 ** -130])
    want = np.array([1.0, 1.0, 1 + 2 ** -7, 1 + 2 ** -6, -2.5, 0.0, 2 ** -130])
    assert np.array_equal(R.bf16(x), want)


def test_conv1d_against_correlate_and_loops():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 3, 17))
    w = rng.normal(size=(4, 3, 5))
    b = rng.normal(size=4)
    # stride 1: sum over input channels of numpy.correlate on the padded row
    y = R.conv1d(x, w, b, 1, 2)
    for bb in range(2):
        for o in range(4):
            ref = b[o] + sum(np.correlate(np.pad(x[bb, c], 2), w[o, c], "valid") for c in range(3))
            assert np.allclose(y[bb, o], ref, rtol=0, atol=1e-12)
    # stride 2: brute force
    y2 = R.conv1d(x, w, b, 2, 2)
    lout = R.conv_out_len(17, 5, 2, 2)
    assert y2.shape == (2, 4, lout)
    for bb in range(2):
        for o in range(4):
            for l in range(lout):
                s = b[o]
                for c in range(3):
                    for t in range(5):
                        i = 2 * l + t - 2
                        if 0 <= i < 17:
                            s += w[o, c, t] * x[bb, c, i]
                assert abs(y2[bb, o, l] - s) < 1e-12


GEOM = {"z0": 0.28, "dz": 0.16, "shift": 2, "T": 24, "cps": 0.05, "J0": 3, "feat": (0.6, 0.3, 0.0, 1.5)}


def test_assembly_brute_force_and_transpose():
    rng = np.random.default_rng(7)
    B, K, Tg = 3, 6, 9
    g = dict(GEOM, T=30)
    G = rng.normal(size=(B * K, Tg))
    qn = rng.normal(size=(B, K))
    rz = rng.uniform([0.1, 0.3], [0.4, 1.2], size=(B, 2))
    out = R.assemble(G, qn, rz, g)
    for b in range(B):
        for i in range(g["T"]):
            s = 0.0
            for k in range(K):
                dz = rz[b, 1] - g["z0"] - k * g["dz"]
                Rr = max(np.hypot(rz[b, 0], dz), 0.5 * g["dz"])
                c = g["shift"] * k + Rr / g["cps"]
                ci = int(np.floor(c))
                f = c - ci
                j = i - ci + g["J0"]
                g0 = G[b * K + k, j] if 0 <= j < Tg else 0.0
                g1 = G[b * K + k, j - 1] if 0 <= j - 1 < Tg else 0.0
                s += qn[b, k] / Rr * ((1 - f) * g0 + f * g1)
            assert abs(out[b, i] - s) < 1e-12
    d = rng.normal(size=(B, g["T"]))
    # the gradient is the exact transpose: <assemble(G), d> = <G, assemble_grad(d)>
    assert abs((out * d).sum() - (G * R.assemble_grad(d, qn, rz, g, Tg)).sum()) < 1e-10
    P = R.pairs(np.array([[0.5, 2.0], [0.7, 3.0]]), 3, 0.28, 0.16)
    assert np.allclose(P, [[0.5, 1.72], [0.5, 1.56], [0.5, 1.40], [0.7, 2.72], [0.7, 2.56], [0.7, 2.40]])


def test_gradients_match_central_differences():
    rng = np.random.default_rng(2)
    K, H, Tg = 8, 16, 20
    p = R.init_params(H, Tg, seed=3)
    for k in p:
        if k.endswith("b"):
            p[k] = rng.normal(scale=0.1, size=p[k].shape)
    B = 2
    qn = rng.uniform(-1, 0, size=(B, K))
    rz = rng.uniform([0.3, 0.5], [0.9, 1.5], size=(B, 2))
    t = rng.normal(size=(B, GEOM["T"]))

    def loss(pp):
        y, _ = R.forward(pp, qn, rz, GEOM, rounding=False)
        return R.mse(y, t)[0]

    y, c = R.forward(p, qn, rz, GEOM, rounding=False)
    g = R.backward(p, c, R.mse(y, t)[1], rounding=False)
    for name in p:
        flat = p[name].reshape(-1)
        idx = rng.choice(flat.size, size=min(8, flat.size), replace=False)
        for i in idx:
            h = 1e-6 * max(1.0, abs(flat[i]))
            old = flat[i]
            flat[i] = old + h
            lp = loss(p)
            flat[i] = old - h
            lm = loss(p)
            flat[i] = old
            num = (lp - lm) / (2 * h)
            ana = g[name].reshape(-1)[i]
            assert abs(num - ana) <= 1e-5 * max(1e-8, abs(num)) + 1e-10, (name, i, num, ana)


def test_adam_first_step_is_a_signed_step():
    rng = np.random.default_rng(4)
    w = rng.normal(size=50)
    gr = rng.normal(size=50)
    w1, m, v = R.adam(w, gr, np.zeros(50), np.zeros(50), 1, lr=1e-3, eps=0.0)
    assert np.allclose(w1, w - 1e-3 * np.sign(gr), rtol=0, atol=1e-15)


def test_feature_and_normalisation_definitions():
    f = R.antenna_features(np.array([[0.6 + 0.15, 5.0 - 2.25]]), 0.6, 0.3, 5.0, 4.5)
    u, v = 0.5, -0.5
    assert abs(f[0, 0] - u) < 1e-14 and abs(f[0, 1] - v) < 1e-14
    assert abs(f[0, 2] - math.sin(math.pi * u)) < 1e-15 and abs(f[0, 5] - math.cos(math.pi * v)) < 1e-15
    assert abs(f[0, 2 + 4 * 14 + 2] - math.sin(15 * math.pi * v)) < 1e-14
    assert np.all(f[0, 62:] == 0)
    qn, s = R.normalize_rows(np.array([[0.0, -2.0, 1.0], [0.0, 0.0, 0.0]]))
    assert np.array_equal(s, [2.0, 0.0]) and np.array_equal(qn, [[0.0, -1.0, 0.5], [0.0, 0.0, 0.0]])


# ---- lattice surrogate reference ------------------------------------------------

def _lattice_case(seed=0, NR=3, D=9, T=40, S=3, K=6, B=5):
    rng = np.random.default_rng(seed)
    G = R.bf16(rng.standard_normal((NR, D, T)))
    q = rng.standard_normal((B, K))
    moff = 4
    ant = np.stack([rng.integers(-1, NR + 1, B), rng.integers(0, 8, B)], axis=1)
    return G, q, ant, S, 2, moff


def test_lattice_forward_brute_force_and_weights():
    """The superposition against one explicit double loop over (k, t), and
    against the product of the profile with the antenna's weight matrix."""
    G, q, ant, S, J, moff = _lattice_case()
    y = R.lattice_forward(G, q, ant, S, J, moff)
    NR, D, T = G.shape
    K = q.shape[1]
    # the same sum written as shifted, zero-padded copies of the table rows
    for b in range(q.shape[0]):
        ir, m = ant[b]
        want = np.zeros(T)
        for k in range(K):
            d = m - k + moff
            if 0 <= ir < NR and 0 <= d < D:
                row = np.concatenate([np.zeros(T + S * K), G[ir, d], np.zeros(T + S * K)])
                lo = T + S * K + J - S * k
                want += q[b, k] * row[lo:lo + T]
        assert np.allclose(y[b], want, rtol=1e-12, atol=1e-12)
    # bin 0 with a lead of J samples: its first J table entries are never used
    assert J > 0
    W = R.lattice_weights(G, ant, K, S, J, moff)
    assert np.allclose(np.einsum("bk,bkt->bt", q, W), y, rtol=1e-12, atol=1e-12)


def test_lattice_gradient_central_differences():
    G, q, ant, S, J, moff = _lattice_case(seed=1)
    rng = np.random.default_rng(2)
    tgt = rng.standard_normal((q.shape[0], G.shape[2]))

    def loss(Gx):
        return 0.5 * ((R.lattice_forward(Gx, q, ant, S, J, moff) - tgt) ** 2).sum()

    dy = R.lattice_forward(G, q, ant, S, J, moff) - tgt
    g = R.lattice_grad(dy, q, ant, S, J, moff, G.shape)
    h = 1e-6
    for idx in [(0, 4, 0), (1, 2, 7), (2, 8, 39), (0, 0, 13), (1, 5, 20)]:
        Gp, Gm = G.copy(), G.copy()
        Gp[idx] += h
        Gm[idx] -= h
        num = (loss(Gp) - loss(Gm)) / (2 * h)
        assert abs(num - g[idx]) <= 1e-6 * (1 + abs(num)), (idx, num, g[idx])
    # entries no antenna reaches have no gradient
    assert np.count_nonzero(g) < g.size
