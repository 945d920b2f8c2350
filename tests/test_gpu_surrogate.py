"""GPU parity of the surrogate kernels (surrogate.h) with the FP64 CPU
reference (oracle/surrogate_ref.py): the tensor-core GEMM in all operand
layouts, the convolutions, the input kernels, Adam, and one full forward +
backward pass of the network; then a short training run on FDTD traces."""
import ctypes as C

import numpy as np
import pytest

import workloads as W
from oracle import surrogate_ref as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    torch.cuda.set_device(0)
    import paper_1001_5341_gb300 as fd
    from paper_1001_5341_gb300 import surrogate as S
    return torch, fd, S


def _p(t):
    return C.c_void_p(t.data_ptr())


def _dev(torch, a, dt=None):
    return torch.tensor(np.asarray(a), dtype=dt or torch.float32, device="cuda")


def _host(t):
    import torch
    return t.detach().to(torch.float64).cpu().numpy()


@pytest.mark.parametrize("ak,bk", [(1, 1), (1, 0), (0, 1), (0, 0)])
@pytest.mark.parametrize("M,N,K", [(70, 50, 40), (129, 200, 2112), (4, 1024, 1024)])
def test_gemm_all_layouts(env, ak, bk, M, N, K):
    torch, fd, S = env
    rng = np.random.default_rng(M + N + K + 2 * ak + bk)
    a = R.bf16(rng.normal(size=(M, K)))
    b = R.bf16(rng.normal(size=(N, K)))
    bias = rng.normal(size=N)
    ref = np.maximum(a @ b.T + bias, 0.0)
    A = _dev(torch, a if ak else a.T.copy(), torch.bfloat16)
    Bm = _dev(torch, b if bk else b.T.copy(), torch.bfloat16)
    ldy = N + 3
    Y = torch.zeros(M, ldy, dtype=torch.float32, device="cuda")
    Yb = torch.zeros(M, ldy, dtype=torch.bfloat16, device="cuda")
    rc = fd.sur_gemm_bf16(_p(A), K if ak else M, ak, _p(Bm), K if bk else N, bk, _p(Y), ldy, _p(Yb), M, N, K,
                          _p(_dev(torch, bias)), 1, 0, None)
    assert rc == 0
    torch.cuda.synchronize()
    y = _host(Y)[:, :N]
    assert np.abs(y - ref).max() <= 2e-5 * np.abs(ref).max()
    assert np.all(_host(Y)[:, N:] == 0)
    assert np.array_equal(_host(Yb)[:, :N], R.bf16(y))
    # accumulate: Y += A B^T (no bias, no relu)
    rc = fd.sur_gemm_bf16(_p(A), K if ak else M, ak, _p(Bm), K if bk else N, bk, _p(Y), ldy, None, M, N, K,
                          None, 0, 1, None)
    assert rc == 0
    torch.cuda.synchronize()
    assert np.abs(_host(Y)[:, :N] - (y + a @ b.T)).max() <= 4e-5 * np.abs(ref).max()


def test_gemm_rejects_bad_sizes(env):
    torch, fd, S = env
    x = torch.zeros(16, dtype=torch.bfloat16, device="cuda")
    y = torch.zeros(16, dtype=torch.float32, device="cuda")
    assert fd.sur_gemm_bf16(_p(x), 4, 1, _p(x), 4, 1, _p(y), 4, None, 4, 4, 0, None, 0, 0, None) == -1
    assert fd.sur_gemm_bf16(_p(x), 2, 1, _p(x), 4, 1, _p(y), 4, None, 4, 4, 4, None, 0, 0, None) == -1
    assert fd.sur_gemm_bf16(None, 4, 1, _p(x), 4, 1, _p(y), 4, None, 4, 4, 4, None, 0, 0, None) == -1


@pytest.mark.parametrize("cin,cout,lin,k,s,pad", [(1, 32, 128, 5, 1, 2), (32, 64, 128, 5, 2, 2), (3, 5, 19, 5, 2, 2)])
def test_conv_forward_and_backward(env, cin, cout, lin, k, s, pad):
    torch, fd, S = env
    rng = np.random.default_rng(cin * 7 + cout)
    B = 5
    x = rng.normal(size=(B, cin, lin)).astype(np.float32).astype(np.float64)
    w = R.bf16(rng.normal(size=(cout, cin, k)) * 0.3)
    b = rng.normal(size=cout).astype(np.float32).astype(np.float64)
    lout = R.conv_out_len(lin, k, s, pad)
    y_ref = np.maximum(R.conv1d(x, w, b, s, pad), 0.0)
    X, Wt, Bt = _dev(torch, x), _dev(torch, w, torch.bfloat16), _dev(torch, b)
    Y = torch.empty(B, cout, lout, dtype=torch.float32, device="cuda")
    assert fd.sur_conv1d_fwd(_p(X), cin * lin, _p(Wt), _p(Bt), _p(Y), B, cin, lin, cout, k, s, pad, 1, None) == 0
    torch.cuda.synchronize()
    assert np.abs(_host(Y) - y_ref).max() <= 1e-5 * np.abs(y_ref).max()
    dy = rng.normal(size=(B, cout, lout)).astype(np.float32).astype(np.float64)
    dz = dy * (_host(Y) > 0)
    dx_ref, dw_ref, db_ref = R.conv1d_grads(x, w, dz, s, pad)
    DX = torch.empty(B, cin, lin, dtype=torch.float32, device="cuda")
    DW = torch.empty(cout, cin, k, dtype=torch.float32, device="cuda")
    DB = torch.empty(cout, dtype=torch.float32, device="cuda")
    assert fd.sur_conv1d_bwd(_p(X), cin * lin, _p(Wt), _p(Y), _p(_dev(torch, dy)), cout * lout, _p(DX), _p(DW),
                             _p(DB), B, cin, lin, cout, k, s, pad, None) == 0
    torch.cuda.synchronize()
    for got, ref in ((DX, dx_ref), (DW, dw_ref), (DB, db_ref)):
        assert np.abs(_host(got) - ref).max() <= 1e-4 * max(np.abs(ref).max(), 1e-6)


def test_input_kernels_and_adam(env):
    torch, fd, S = env
    rng = np.random.default_rng(5)
    B = 37
    q = -rng.uniform(0, 3, size=(B, 128))
    q[3] = 0.0
    qn_ref, s_ref = R.normalize_rows(q)
    Q = _dev(torch, q)
    QN = torch.empty(B, 128, dtype=torch.float32, device="cuda")
    Sv = torch.empty(B, dtype=torch.float32, device="cuda")
    assert fd.sur_normalize_rows(_p(Q), B, 128, _p(QN), _p(Sv), None) == 0
    rz = rng.uniform([0.3, 0.5], [0.9, 9.5], size=(B, 2))
    F = torch.empty(B, 64, dtype=torch.float32, device="cuda")
    assert fd.sur_antenna_features(_p(_dev(torch, rz)), B, *S.Geometry().feat, _p(F), None) == 0
    Y = _dev(torch, rng.normal(size=(B, 10)))
    y0 = _host(Y)
    assert fd.sur_scale_rows(_p(Y), B, 10, _p(Sv), 2.0, 0, None) == 0
    torch.cuda.synchronize()
    assert np.allclose(_host(QN), qn_ref, rtol=1e-6, atol=1e-7)
    assert np.allclose(_host(Sv), s_ref, rtol=1e-6)
    assert np.abs(_host(F) - R.antenna_features(rz, *S.Geometry().feat)).max() < 2e-5
    assert np.allclose(_host(Y), y0 * 2.0 * s_ref[:, None], rtol=1e-6, atol=1e-7)
    assert fd.sur_scale_rows(_p(Y), B, 10, _p(Sv), 0.5, 1, None) == 0
    torch.cuda.synchronize()
    assert np.allclose(_host(Y), np.where(s_ref[:, None] > 0, y0, 0.0), rtol=1e-5, atol=1e-6)
    # Adam, three steps
    n = 1000
    w, g = rng.normal(size=n), rng.normal(size=(3, n))
    Wt, Wb = _dev(torch, w), torch.empty(n, dtype=torch.bfloat16, device="cuda")
    Mt, Vt = torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    m, v, wr = np.zeros(n), np.zeros(n), w.astype(np.float32).astype(np.float64)
    for t in range(3):
        assert fd.sur_adam(_p(Wt), _p(Wb), _p(_dev(torch, g[t])), _p(Mt), _p(Vt), n, 1e-2, 0.9, 0.999, 1e-8, t + 1,
                           None) == 0
        wr, m, v = R.adam(wr, g[t].astype(np.float32).astype(np.float64), m, v, t + 1, 1e-2)
    torch.cuda.synchronize()
    assert np.abs(_host(Wt) - wr).max() < 1e-5
    assert np.array_equal(_host(Wb), R.bf16(_host(Wt)))


def test_pairs_and_assembly(env):
    torch, fd, S = env
    rng = np.random.default_rng(8)
    B, K, Tg, T = 5, 37, 60, 90
    g = {"z0": 0.28, "dz": 0.08, "shift": 3, "T": T, "cps": 0.0119, "J0": 5}
    rz = rng.uniform([0.1, 0.5], [0.5, 3.0], size=(B, 2))
    RZ = _dev(torch, rz)
    P = torch.empty(B * K, 2, dtype=torch.float32, device="cuda")
    assert fd.sur_pairs(_p(RZ), B, K, g["z0"], g["dz"], _p(P), None) == 0
    G = rng.normal(size=(B * K, Tg))
    qn = rng.normal(size=(B, K))
    Y = torch.empty(B, T, dtype=torch.float32, device="cuda")
    assert fd.sur_assemble(_p(_dev(torch, G)), _p(_dev(torch, qn)), _p(RZ), B, K, Tg, g["shift"], T, g["z0"],
                           g["dz"], g["cps"], g["J0"], _p(Y), None) == 0
    d = rng.normal(size=(B, T))
    DG = torch.empty(B * K, Tg, dtype=torch.float32, device="cuda")
    DGb = torch.empty(B * K, Tg, dtype=torch.bfloat16, device="cuda")
    assert fd.sur_assemble_bwd(_p(_dev(torch, d)), _p(_dev(torch, qn)), _p(RZ), B, K, Tg, g["shift"], T, g["z0"],
                               g["dz"], g["cps"], g["J0"], _p(DG), _p(DGb), None) == 0
    torch.cuda.synchronize()
    rz32 = rz.astype(np.float32).astype(np.float64)
    assert np.abs(_host(P) - R.pairs(rz32, K, g["z0"], g["dz"])).max() < 2e-6
    y_ref = R.assemble(G, qn, rz32, g)
    assert np.linalg.norm(_host(Y) - y_ref) <= 1e-4 * np.linalg.norm(y_ref)
    dg_ref = R.assemble_grad(d, qn, rz32, g, Tg)
    assert np.linalg.norm(_host(DG) - dg_ref) <= 1e-4 * np.linalg.norm(dg_ref)
    assert np.array_equal(_host(DGb), R.bf16(_host(DG)))


def test_network_step_matches_reference(env):
    """One forward + backward pass of the whole network, GPU kernels against
    the CPU reference with the same bf16 weights and rounding points."""
    torch, fd, S = env
    rng = np.random.default_rng(6)
    geo = S.Geometry(K=40, z0=0.28, dz=0.0822, shift=4, T=160, Tg=160, cps=0.0119, J0=8)
    net = S.Net(geo, hidden=256, seed=11)
    for k in net.p:   # non-zero biases so every term is exercised
        if k.endswith("b"):
            net.p[k].copy_(_dev(torch, rng.normal(scale=0.05, size=tuple(net.p[k].shape))))
    B = 6
    q = -rng.uniform(0, 1, size=(B, geo.K)) * 1e-9
    rz = rng.uniform([0.3, 0.5], [0.9, 3.5], size=(B, 2))
    tgt = rng.normal(size=(B, geo.T))
    y = net.forward(_dev(torch, q), _dev(torch, rz), scale_out=False)
    net._workspace(B)["tn"].copy_(_dev(torch, tgt))
    net.backward(B)
    torch.cuda.synchronize()
    p = {k: (_host(net.pb[k]) if k in net.pb else _host(net.p[k])) for k in net.p}
    qn, _ = R.normalize_rows(q.astype(np.float32).astype(np.float64))
    gd = {"z0": geo.z0, "dz": geo.dz, "shift": geo.shift, "T": geo.T, "cps": geo.cps, "J0": geo.J0,
          "feat": geo.feat}
    y_ref, cache = R.forward(p, qn, rz.astype(np.float32).astype(np.float64), gd)
    g_ref = R.backward(p, cache, R.mse(y_ref, tgt.astype(np.float32).astype(np.float64))[1])

    def rel(a, b):
        return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)

    assert rel(_host(y), y_ref) < 1e-3
    for k in g_ref:
        assert rel(_host(net.g[k]), g_ref[k]) < 5e-3, k


def test_training_on_fdtd_traces_beats_the_mean_trace(env):
    """A short run of the whole pipeline: FDTD traces of a small grid (48
    showers, 32 antennas each), 3000 optimiser steps, and traces of 8
    held-out showers predicted far better than by the training set's mean
    normalised trace (the best a fixed template does without the network)."""
    torch, fd, S = env
    grid = W.surrogate_grid(nx=64, ny=64, nz=256, steps=640, n_bins=56)
    runs = W.surrogate_runs(seed=21, n_runs=48, n_probes=32, grid=grid, r_range=(0.15, 0.4),
                            z_range=(0.4, 4.6), z1_range=(0.2, 1.0), len_range=(0.5, 1.8))
    data = S.generate(grid, runs, decim=1)
    geo = S.Geometry.of(grid, decim=1, m=8, feat=(0.275, 0.125, 0.0, 5.0))
    N = data.trace.shape[0]
    assert N == 48 * 32 and data.trace.shape[1] == geo.T == 640
    ntr = 40 * 32
    tr = _host(data.trace)
    s = np.abs(_host(data.q)).max(axis=1)
    c_out = float(np.sqrt(np.mean((tr[:ntr] / s[:ntr, None]) ** 2)))
    net = S.Net(geo, hidden=512, seed=3, c_out=c_out)
    rng = np.random.default_rng(0)
    for it in range(3000):
        idx = torch.tensor(rng.choice(ntr, size=32, replace=False), device="cuda")
        net.train_batch(data.q[idx].contiguous(), data.rz[idx].contiguous(), data.trace[idx].contiguous(),
                        lr=1e-3 if it < 2000 else 2e-4)
    pred = _host(net.predict(data.q[ntr:], data.rz[ntr:]))
    err = S.rel_l2(pred, tr[ntr:])
    mean_tmpl = np.mean(tr[:ntr] / s[:ntr, None], axis=0)
    err_mean = S.rel_l2(mean_tmpl[None, :] * s[ntr:, None], tr[ntr:])
    assert np.median(err) < 0.6 * np.median(err_mean), (np.median(err), np.median(err_mean))


# ---- lattice surrogate ------------------------------------------------------------

def _lattice_case(torch, seed=3, NR=4, D=30, T=300, S=4, K=20, B=9):
    rng = np.random.default_rng(seed)
    G = R.bf16(rng.standard_normal((NR, D, T)) * 0.1)
    q = rng.standard_normal((B, K))
    q[:, ::3] = 0.0
    moff = K - 1
    ant = np.stack([rng.integers(-1, NR + 1, B), rng.integers(0, D - K + 1, B)], axis=1).astype(np.int32)
    return G, q, ant, S, S, moff


def test_lattice_kernels_match_reference(env):
    torch, fd, S = env
    G, q, ant, Ss, J, moff = _lattice_case(torch)
    NR, D, T = G.shape
    B, K = q.shape
    Gb = _dev(torch, G, torch.bfloat16)
    qd, ad = _dev(torch, q), _dev(torch, ant, torch.int32)
    y = torch.empty(B, T, dtype=torch.float32, device="cuda")
    fd.check(fd.sur_lattice_fwd(_p(Gb), None, _p(qd), _p(ad), B, K, NR, D, T, Ss, J, moff, _p(y), None), "fwd")
    want = R.lattice_forward(G, q.astype(np.float32).astype(np.float64), ant, Ss, J, moff)
    assert np.abs(_host(y) - want).max() <= 1e-5 * np.abs(want).max()
    # f32 table, and a bf16 part + remainder pair that carries it to ~2^-17
    Gf = np.random.default_rng(5).standard_normal(G.shape).astype(np.float32).astype(np.float64)
    Gfd = _dev(torch, Gf)
    fd.check(fd.sur_lattice_fwd_f32(_p(Gfd), _p(qd), _p(ad), B, K, NR, D, T, Ss, J, moff, _p(y), None), "f32")
    want = R.lattice_forward(Gf, q.astype(np.float32).astype(np.float64), ant, Ss, J, moff)
    assert np.abs(_host(y) - want).max() <= 1e-5 * np.abs(want).max()
    hi = torch.empty(G.shape, dtype=torch.bfloat16, device="cuda")
    lo = torch.empty(G.shape, dtype=torch.bfloat16, device="cuda")
    fd.check(fd.sur_split_bf16(_p(Gfd), _p(hi), _p(lo), Gf.size, None), "split")
    assert np.array_equal(_host(hi), R.bf16(Gf))
    assert np.array_equal(_host(lo), R.bf16(Gf.astype(np.float32) - R.bf16(Gf).astype(np.float32)))
    assert np.abs(_host(hi) + _host(lo) - Gf).max() <= 2.0 ** -16 * np.abs(Gf).max()
    fd.check(fd.sur_lattice_fwd(_p(hi), _p(lo), _p(qd), _p(ad), B, K, NR, D, T, Ss, J, moff, _p(y), None), "pair")
    assert np.abs(_host(y) - want).max() <= 3e-5 * np.abs(want).max()
    dy = np.random.default_rng(4).standard_normal((B, T))
    dG = torch.zeros(NR, D, T, dtype=torch.float32, device="cuda")
    fd.check(fd.sur_lattice_bwd(_p(_dev(torch, dy)), _p(qd), _p(ad), B, K, NR, D, T, Ss, J, moff, _p(dG), None),
             "bwd")
    gw = R.lattice_grad(dy, q.astype(np.float32).astype(np.float64), ant, Ss, J, moff, G.shape)
    assert np.abs(_host(dG) - gw).max() <= 1e-5 * np.abs(gw).max()
    W = torch.empty(B, K, T, dtype=torch.bfloat16, device="cuda")
    fd.check(fd.sur_lattice_weights(_p(Gb), _p(ad), B, K, NR, D, T, Ss, J, moff, _p(W), None), "weights")
    assert np.array_equal(_host(W), R.lattice_weights(G, ant, K, Ss, J, moff))
    assert fd.sur_lattice_fwd(None, None, _p(qd), _p(ad), B, K, NR, D, T, Ss, J, moff, _p(y), None) == -1
    # the K-major weights of the tcgen05 GEMM: W3[a][t][koff + k], other columns untouched
    KP = (3 * K + 7) // 8 * 8
    W3 = torch.full((B, T, KP), 7.0, dtype=torch.bfloat16, device="cuda")
    fd.check(fd.sur_lattice_weights_kmajor(_p(Gb), _p(ad), B, K, NR, D, T, Ss, J, moff, _p(W3), KP, K, None), "wk")
    w3 = _host(W3)
    assert np.array_equal(w3[:, :, K:2 * K], R.lattice_weights(G, ant, K, Ss, J, moff).transpose(0, 2, 1))
    assert np.all(w3[:, :, :K] == 7.0) and np.all(w3[:, :, 2 * K:] == 7.0)
    assert fd.sur_lattice_weights_kmajor(_p(Gb), _p(ad), B, K, NR, D, T, Ss, J, moff, _p(W3), 2 * K - 1, K,
                                         None) == -1
    # the split profile rows [hi, hi, lo, 0 ...]
    Q3 = torch.full((B, KP), 7.0, dtype=torch.bfloat16, device="cuda")
    fd.check(fd.sur_split3_bf16(_p(qd), B, K, _p(Q3), KP, None), "split3")
    q32 = q.astype(np.float32)
    hi_q, q3 = R.bf16(q32), _host(Q3)
    assert np.array_equal(q3[:, :K], hi_q) and np.array_equal(q3[:, K:2 * K], hi_q)
    assert np.array_equal(q3[:, 2 * K:3 * K], R.bf16(q32 - hi_q.astype(np.float32)))
    assert np.all(q3[:, 3 * K:] == 0)
    assert fd.sur_split3_bf16(_p(qd), B, K, _p(Q3), 3 * K - 1, None) == -1


@pytest.mark.parametrize("M,N,K", [(70, 50, 40), (129, 200, 2112), (300, 1024, 96), (1000, 384, 256),
                                   (4, 1024, 1024), (257, 130, 30)])
def test_gemm_tcgen05_layouts(env, M, N, K):
    """Both operand layouts of the tcgen05 kernel (128-byte swizzled slices,
    unswizzled core matrices) against the FP64 product of the same bf16
    operands, with the fused epilogue; K not a multiple of 8 reads zeros past
    K on the swizzled path; the mma.sync kernel agrees; the launch counter
    shows which kernel ran; no pipeline wait gave up."""
    torch, fd, S = env
    rng = np.random.default_rng(M * 7 + N + K)
    lda = (K + 7) // 8 * 8
    a = R.bf16(rng.normal(size=(M, K)))
    b = R.bf16(rng.normal(size=(N, K)))
    bias = rng.normal(size=N)
    ref = np.maximum(a @ b.T + bias, 0.0)
    A = torch.zeros(M, lda, dtype=torch.bfloat16, device="cuda")
    Bm = torch.zeros(N, lda, dtype=torch.bfloat16, device="cuda")
    A[:, :K] = _dev(torch, a, torch.bfloat16)
    Bm[:, :K] = _dev(torch, b, torch.bfloat16)
    # garbage past K in the padding: only the first K columns may count
    A[:, K:] = 3.0
    Bm[:, K:] = -5.0
    bd = _dev(torch, bias)
    ldy = N + 5
    outs = {}
    try:
        for path in (2, 3, 1):
            if path == 3 and K % 8:
                assert fd.sur_gemm_set_path(3) == 0
                Y = torch.zeros(M, ldy, dtype=torch.float32, device="cuda")
                assert fd.sur_gemm_bf16(_p(A), lda, 1, _p(Bm), lda, 1, _p(Y), ldy, None, M, N, K, _p(bd), 1, 0,
                                        None) == -1
                continue
            assert fd.sur_gemm_set_path(path) == 0
            n0 = fd.sur_gemm_tc_launches()
            Y = torch.zeros(M, ldy, dtype=torch.float32, device="cuda")
            Yb = torch.zeros(M, ldy, dtype=torch.bfloat16, device="cuda")
            rc = fd.sur_gemm_bf16(_p(A), lda, 1, _p(Bm), lda, 1, _p(Y), ldy, _p(Yb), M, N, K, _p(bd), 1, 0, None)
            assert rc == 0
            torch.cuda.synchronize()
            assert fd.sur_gemm_tc_launches() - n0 == (0 if path == 1 else 1)
            y = _host(Y)
            assert np.abs(y[:, :N] - ref).max() <= 2e-5 * np.abs(ref).max(), path
            assert np.all(y[:, N:] == 0)
            assert np.array_equal(_host(Yb)[:, :N], R.bf16(y[:, :N]))
            outs[path] = y[:, :N]
            if path == 2:   # accumulate into Y, no bias, no ReLU
                fd.check(fd.sur_gemm_bf16(_p(A), lda, 1, _p(Bm), lda, 1, _p(Y), ldy, None, M, N, K, None, 0, 1,
                                          None), "acc")
                torch.cuda.synchronize()
                assert np.abs(_host(Y)[:, :N] - (y[:, :N] + a @ b.T)).max() <= 4e-5 * np.abs(ref).max()
        assert fd.sur_gemm_tc_failed() == 0
        assert np.abs(outs[1] - outs[2]).max() <= 2e-5 * np.abs(ref).max()
        # an MN-major operand is not the tcgen05 kernel's: rejected when it alone was asked for
        assert fd.sur_gemm_set_path(2) == 0
        Y = torch.zeros(M, ldy, dtype=torch.float32, device="cuda")
        assert fd.sur_gemm_bf16(_p(A), lda, 1, _p(Bm), N, 0, _p(Y), ldy, None, M, N, min(K, N), None, 0, 0,
                                None) == -1
    finally:
        assert fd.sur_gemm_set_path(0) == 0
    # the automatic choice: K-major operands with 16-byte rows take the tcgen05 kernel, others mma.sync
    n0 = fd.sur_gemm_tc_launches()
    Y = torch.zeros(M, ldy, dtype=torch.float32, device="cuda")
    fd.check(fd.sur_gemm_bf16(_p(A), lda, 1, _p(Bm), lda, 1, _p(Y), ldy, None, M, N, K, None, 0, 0, None), "auto")
    assert fd.sur_gemm_tc_launches() == n0 + 1
    if K % 8:
        At = _dev(torch, a, torch.bfloat16)
        fd.check(fd.sur_gemm_bf16(_p(At), K, 1, _p(Bm), lda, 1, _p(Y), ldy, None, M, N, K, None, 0, 0, None), "mma")
        assert fd.sur_gemm_tc_launches() == n0 + 1
    assert fd.sur_gemm_set_path(4) == -1


@pytest.mark.parametrize("shared_a", [True, False])
def test_gemm_tcgen05_batched(env, shared_a):
    """Batched products in one launch (an operand shared by the batch or
    strided), the row scale and alpha fused into the epilogue, against the
    FP64 products of the same bf16 operands; argument checks."""
    torch, fd, S = env
    M, N, K, nb = 200, 300, 93, 5
    lda = 96
    rng = np.random.default_rng(11 + shared_a)
    a = R.bf16(rng.normal(size=(1 if shared_a else nb, M, K)))
    b = R.bf16(rng.normal(size=(nb, N, K)))
    rs = rng.uniform(0.5, 2.0, size=M)
    alpha = 0.37
    A = torch.zeros(a.shape[0], M, lda, dtype=torch.bfloat16, device="cuda")
    Bm = torch.zeros(nb, N, lda, dtype=torch.bfloat16, device="cuda")
    A[:, :, :K] = _dev(torch, a, torch.bfloat16)
    Bm[:, :, :K] = _dev(torch, b, torch.bfloat16)
    ldy = N + 4
    Y = torch.full((nb, M, ldy), 9.0, dtype=torch.float32, device="cuda")
    rsd = _dev(torch, rs)
    n0 = fd.sur_gemm_tc_launches()
    rc = fd.sur_gemm_bf16_batched(_p(A), lda, 0 if shared_a else M * lda, _p(Bm), lda, N * lda, _p(Y), ldy, M * ldy,
                                  M, N, K, nb, _p(rsd), C.c_float(alpha), None)
    assert rc == 0
    torch.cuda.synchronize()
    assert fd.sur_gemm_tc_launches() == n0 + 1
    y = _host(Y)
    for z in range(nb):
        az = a[0 if shared_a else z]
        ref = alpha * np.float32(rs)[:, None].astype(np.float64) * (az @ b[z].T)
        assert np.abs(y[z, :, :N] - ref).max() <= 2e-5 * np.abs(ref).max(), z
        assert np.all(y[z, :, N:] == 9.0)
    assert fd.sur_gemm_tc_failed() == 0
    args = [_p(A), lda, 0, _p(Bm), lda, N * lda, _p(Y), ldy, M * ldy, M, N, K, nb, None, C.c_float(1.0), None]
    bad = list(args); bad[1] = 93                  # lda not a multiple of 8
    assert fd.sur_gemm_bf16_batched(*bad) == -1
    bad = list(args); bad[8] = M * ldy - 1         # output batches overlap
    assert fd.sur_gemm_bf16_batched(*bad) == -1
    bad = list(args); bad[12] = 0                  # empty batch
    assert fd.sur_gemm_bf16_batched(*bad) == -1
    try:
        assert fd.sur_gemm_set_path(1) == 0        # mma.sync only: no batched form
        assert fd.sur_gemm_bf16_batched(*args) == -1
    finally:
        assert fd.sur_gemm_set_path(0) == 0


def test_lattice_surrogate_learns_held_out_showers(env):
    """A small version of the lattice surrogate (64x64x256 grid, c dt = dx/2,
    bins of 8 steps, antennas at r = 0.20-0.36 m): trained by the library's
    kernels on 24 FDTD showers, it predicts 6 held-out showers at every lattice
    antenna to a median relative L2 below 2 %, far below the method without
    the network (each antenna's mean normalised trace), and its GEMM path
    agrees with its gather path."""
    torch, fd, S = env
    grid = W.surrogate_lattice_grid(nx=64, ny=64, nz=256, npml=8, steps=768, n_bins=56)
    ir, m, xyz = W.surrogate_lattice_antennas(grid, r_range=(0.2, 0.36), z_range=(0.4, 4.6))
    runs = lambda seed, n: W.surrogate_runs(seed=seed, n_runs=n, n_probes=1, grid=grid, z1_range=(0.3, 1.2),
                                            len_range=(0.6, 1.8), r_range=(0.2, 0.3), z_range=(0.5, 4.5))
    train = S.generate_lattice(grid, runs(71, 24), ir, m, xyz)
    test = S.generate_lattice(grid, runs(72, 6), ir, m, xyz)
    geo = S.LatticeGeometry.of(grid, ir, m)
    net = S.train_lattice(train, geo, steps=20000, batch=512, lr=3e-3, seed=1)
    Rn, A = test.q.shape[0], len(ir)
    qq, aa = test.q.repeat_interleave(A, dim=0), test.ant.repeat(Rn, 1)
    ref = _host(test.trace.reshape(Rn * A, -1))
    err = S.rel_l2(_host(net.predict(qq, aa)), ref)
    tmpl = (train.trace / train.q.abs().amax(dim=1)[:, None, None]).mean(dim=0)
    base = _host((test.q.abs().amax(dim=1)[:, None, None] * tmpl[None]).reshape(Rn * A, -1))
    err0 = S.rel_l2(base, ref)
    print(f"\nlattice surrogate held-out median {np.median(err):.2e} p90 {np.percentile(err, 90):.2e}; "
          f"mean-trace baseline median {np.median(err0):.2e}")
    assert np.median(err) <= 0.01
    assert np.median(err) <= 0.05 * np.median(err0)
    yg = net.predict_grid(test.q[:3].contiguous(), test.ant[:5].contiguous())
    yf = net.predict(test.q[:3].repeat_interleave(5, dim=0).contiguous(), test.ant[:5].repeat(3, 1).contiguous())
    d = S.rel_l2(_host(yg.permute(1, 0, 2).reshape(15, -1)), _host(yf))
    assert np.median(d) <= 1e-4
