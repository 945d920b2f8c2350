"""FP64 NumPy reference of the learned near-field surrogate (forward, backward,
Adam) -- TEST INFRASTRUCTURE.

Only tests/ and bench.py's reference legs may import this module.  It shares
no code with the CUDA kernels (paper_1001_5341_gb300/csrc/surrogate.cu); it
states the same network from its definition.

The trace at an antenna is linear in the shower's binned charge profile q_k
(the field equations are linear in the current, Sec. III.A), and in a uniform
medium the response of bin k depends only on the antenna's radius r and its
axial offset dz = z_a - z_k and on the time since the shower front reached
the bin.  With bins of m shower steps (bin length m v dt) that time is a
whole number of samples, shift k, so

    trace[i] = peak|q| c_out sum_k qn_k (1/R_k) G(r, dz_k)(i - shift k - R_k/c'),

qn = q / peak|q|, R_k the antenna's distance from bin k: each response sits
in its own retarded time (linear interpolation between samples), and G(r, dz)
is a waveform of Tg samples (J0 of them before the direct arrival) from an
MLP:
    64 features of (r, dz) -> H ReLU -> H ReLU -> Tg.
This is the learned counterpart of the Green's function superposition of
Sec. II.  Precision mirrors the GPU path: the values the GPU stores in bf16
(weights, the MLP inputs and activations, the gradients fed to the
tensor-core GEMMs) are rounded to bf16 here at the same points; the rest is
FP64 (the GPU keeps f32).  Rounding is round-to-nearest-even of the float32
value.

The 1D convolution helpers below are the reference of the general conv1d
kernels of the same library.
"""
from __future__ import annotations

import math

import numpy as np

N_FEAT = 64


def bf16(x):
    """Round to bfloat16 (nearest, ties to even) through float32; returns float64."""
    u = np.ascontiguousarray(np.asarray(x, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def conv_out_len(lin, k, stride, pad):
    return (lin + 2 * pad - k) // stride + 1


def conv1d(x, w, b, stride, pad):
    """y[b,o,l] = b[o] + sum_{c,t} w[o,c,t] x[b,c,l*stride+t-pad] (zero outside)."""
    B, cin, lin = x.shape
    cout, _, k = w.shape
    lout = conv_out_len(lin, k, stride, pad)
    xp = np.zeros((B, cin, lin + 2 * pad + k))
    xp[:, :, pad:pad + lin] = x
    y = np.zeros((B, cout, lout))
    for t in range(k):
        cols = xp[:, :, t:t + stride * (lout - 1) + 1:stride]          # [B, cin, lout]
        y += np.einsum("oc,bcl->bol", w[:, :, t], cols)
    return y + b[None, :, None]


def conv1d_grads(x, w, dz, stride, pad):
    """Gradients of conv1d given dz = dL/dy: (dx, dw, db)."""
    B, cin, lin = x.shape
    cout, _, k = w.shape
    lout = dz.shape[2]
    xp = np.zeros((B, cin, lin + 2 * pad + k))
    xp[:, :, pad:pad + lin] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for t in range(k):
        sl = slice(t, t + stride * (lout - 1) + 1, stride)
        dw[:, :, t] = np.einsum("bol,bcl->oc", dz, xp[:, :, sl])
        dxp[:, :, sl] += np.einsum("oc,bol->bcl", w[:, :, t], dz)
    return dxp[:, :, pad:pad + lin], dw, dz.sum(axis=(0, 2))


def antenna_features(rz, r0, rs, z0, zs):
    rz = np.asarray(rz, dtype=np.float64)
    u = (rz[:, 0] - r0) / rs
    v = (rz[:, 1] - z0) / zs
    out = np.zeros((rz.shape[0], N_FEAT))
    out[:, 0] = u
    out[:, 1] = v
    for f in range(1, 16):
        c = 2 + 4 * (f - 1)
        out[:, c] = np.sin(f * math.pi * u)
        out[:, c + 1] = np.cos(f * math.pi * u)
        out[:, c + 2] = np.sin(f * math.pi * v)
        out[:, c + 3] = np.cos(f * math.pi * v)
    return out


def normalize_rows(q):
    q = np.asarray(q, dtype=np.float64)
    s = np.abs(q).max(axis=1)
    inv = np.where(s > 0, 1.0 / np.where(s > 0, s, 1.0), 0.0)
    return q * inv[:, None], s


def pairs(rz, K, z0, dz):
    """[B*K, 2]: (r_b, z_b - z0 - k dz) for every antenna b and bin k."""
    rz = np.asarray(rz, dtype=np.float64)
    B = rz.shape[0]
    out = np.zeros((B * K, 2))
    out[:, 0] = np.repeat(rz[:, 0], K)
    out[:, 1] = (rz[:, 1][:, None] - z0 - np.arange(K)[None, :] * dz).reshape(-1)
    return out


def placement(rz, K, g):
    """Retarded-time placement of bin k's response at antenna b: integer
    offset ci, interpolation weight f and amplitude 1/R, with R the distance
    from the antenna to bin k (floored at dz/2) and the offset shift k + R/cps
    samples."""
    rz = np.asarray(rz, dtype=np.float64)
    r = rz[:, 0][:, None]
    d = rz[:, 1][:, None] - g["z0"] - np.arange(K)[None, :] * g["dz"]
    R = np.maximum(np.sqrt(r * r + d * d), 0.5 * g["dz"])
    c = g["shift"] * np.arange(K)[None, :] + R / g["cps"]
    ci = np.floor(c).astype(np.int64)
    return ci, c - ci, 1.0 / R


def assemble(G, qn, rz, g):
    """out[b, i] = sum_k qn[b,k] a_bk ((1-f) G[bk, i-ci+J0] + f G[bk, i-ci-1+J0])."""
    B, K = qn.shape
    Tg, T, J0 = G.shape[1], g["T"], g["J0"]
    ci, f, a = placement(rz, K, g)
    out = np.zeros((B, T))
    Gp = np.zeros((B * K, Tg + 1))
    Gp[:, 1:] = G                      # Gp[:, j+1] = G[:, j]; Gp[:, 0] = G[:, -1] = 0
    for b in range(B):
        for k in range(K):
            j = np.arange(T) - ci[b, k] + J0
            g0 = np.where((j >= 0) & (j < Tg), Gp[b * K + k, np.clip(j + 1, 0, Tg)], 0.0)
            g1 = np.where((j - 1 >= 0) & (j - 1 < Tg), Gp[b * K + k, np.clip(j, 0, Tg)], 0.0)
            out[b] += qn[b, k] * a[b, k] * ((1 - f[b, k]) * g0 + f[b, k] * g1)
    return out


def assemble_grad(dout, qn, rz, g, Tg):
    """dG[bk, j] = qn a ((1-f) dout[b, j+ci-J0] + f dout[b, j+ci+1-J0])."""
    B, K = qn.shape
    T, J0 = dout.shape[1], g["J0"]
    ci, f, a = placement(rz, K, g)
    dG = np.zeros((B * K, Tg))
    jj = np.arange(Tg)
    for b in range(B):
        for k in range(K):
            i0 = jj + ci[b, k] - J0
            d0 = np.where((i0 >= 0) & (i0 < T), dout[b, np.clip(i0, 0, T - 1)], 0.0)
            d1 = np.where((i0 + 1 >= 0) & (i0 + 1 < T), dout[b, np.clip(i0 + 1, 0, T - 1)], 0.0)
            dG[b * K + k] = qn[b, k] * a[b, k] * ((1 - f[b, k]) * d0 + f[b, k] * d1)
    return dG


def init_params(H, Tg, seed=0):
    """He-uniform initial weights (f64, to be rounded to bf16 for use)."""
    rng = np.random.default_rng(seed)
    p = {}
    for i, (fin, fout) in enumerate(((N_FEAT, H), (H, H), (H, Tg))):
        lim = math.sqrt(6.0 / fin) if i < 2 else math.sqrt(3.0 / fin)
        p[f"f{i}w"] = rng.uniform(-lim, lim, size=(fout, fin))
        p[f"f{i}b"] = np.zeros(fout)
    return p


def forward(p, qn, rz, geom, rounding=True):
    """Normalised traces [B, T] and the cache for backward.

    p: parameters (pass bf16-rounded weights); qn: [B, K] normalised profiles;
    rz: [B, 2] antenna (r, z); geom: dict z0, dz, shift, T, cps, J0 and the
    feature scaling feat = (r0, rs, z0f, zsf)."""
    R = bf16 if rounding else (lambda a: np.asarray(a, dtype=np.float64))
    B, K = qn.shape
    P = pairs(rz, K, geom["z0"], geom["dz"])
    Fb = R(antenna_features(P, *geom["feat"]))
    h1 = np.maximum(Fb @ p["f0w"].T + p["f0b"], 0.0)
    h1b = R(h1)
    h2 = np.maximum(h1b @ p["f1w"].T + p["f1b"], 0.0)
    h2b = R(h2)
    G = h2b @ p["f2w"].T + p["f2b"]
    y = assemble(G, qn, rz, geom)
    return y, {"qn": qn, "rz": rz, "Fb": Fb, "h1": h1, "h1b": h1b, "h2": h2, "h2b": h2b, "G": G, "geom": geom}


def mse(y, t):
    n = y.size
    return float(((y - t) ** 2).sum() / n), 2.0 * (y - t) / n


def backward(p, c, dy, rounding=True):
    """Gradients of every parameter given dL/dy (normalised traces)."""
    R = bf16 if rounding else (lambda a: np.asarray(a, dtype=np.float64))
    g = {}
    dG = assemble_grad(dy, c["qn"], c["rz"], c["geom"], p["f2w"].shape[0])
    dGb = R(dG)
    g["f2w"] = dGb.T @ c["h2b"]
    g["f2b"] = dG.sum(axis=0)
    dz2 = (dGb @ p["f2w"]) * (c["h2"] > 0)
    dz2b = R(dz2)
    g["f1w"] = dz2b.T @ c["h1b"]
    g["f1b"] = dz2.sum(axis=0)
    dz1 = (dz2b @ p["f1w"]) * (c["h1"] > 0)
    dz1b = R(dz1)
    g["f0w"] = dz1b.T @ c["Fb"]
    g["f0b"] = dz1.sum(axis=0)
    return g


def adam(w, gr, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * gr
    v = b2 * v + (1 - b2) * gr * gr
    w = w - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    return w, m, v


# ---- lattice surrogate ----------------------------------------------------------
#
# With the shower moving half a cell per step and bins of 2S steps (S trace
# samples of two steps), the field of bin k at an antenna equals the field of
# bin 0 at the antenna moved S k cells back along z, S k samples earlier (the
# exact translation property pinned in tests/test_oracle_source.py).  The
# trace is linear in the profile, so for an antenna of radial class ir at the
# start of bin m:
#     y[t] = sum_k q[k] G[ir][m - k + moff][t - S k + J]   (0 <= t - S k + J < T),
# with G the learned response of one bin and J lead samples.  Plain loops
# over the definition.

def lattice_forward(G, q, ant, S, J, moff):
    """y [B][T] from G [NR][D][T] (values as stored), q [B][K], ant [B][2]."""
    NR, D, T = G.shape
    B, K = q.shape
    y = np.zeros((B, T))
    for b in range(B):
        ir, m = int(ant[b][0]), int(ant[b][1])
        if not 0 <= ir < NR:
            continue
        for k in range(K):
            d = m - k + moff
            if not 0 <= d < D:
                continue
            for t in range(T):
                tau = t - S * k + J
                if 0 <= tau < T:
                    y[b, t] += q[b, k] * G[ir, d, tau]
    return y


def lattice_grad(dy, q, ant, S, J, moff, shape):
    """dL/dG [NR][D][T] for dL/dy = dy [B][T]: the transpose of lattice_forward."""
    NR, D, T = shape
    B, K = q.shape
    g = np.zeros(shape)
    for b in range(B):
        ir, m = int(ant[b][0]), int(ant[b][1])
        if not 0 <= ir < NR:
            continue
        for k in range(K):
            d = m - k + moff
            if not 0 <= d < D:
                continue
            for t in range(T):
                tau = t - S * k + J
                if 0 <= tau < T:
                    g[ir, d, tau] += q[b, k] * dy[b, t]
    return g


def lattice_weights(G, ant, K, S, J, moff):
    """W [A][K][T]: W[a][k][t] = G[ir][m - k + moff][t - S k + J] (0 elsewhere)."""
    NR, D, T = G.shape
    W = np.zeros((len(ant), K, T))
    for a, (ir, m) in enumerate(ant):
        for k in range(K):
            d = int(m) - k + moff
            if not (0 <= int(ir) < NR and 0 <= d < D):
                continue
            for t in range(T):
                tau = t - S * k + J
                if 0 <= tau < T:
                    W[a, k, t] = G[int(ir), d, tau]
    return W
