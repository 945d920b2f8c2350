"""GPU adjoint (fdtd_adjoint_step, fdtd_adjoint_gradient, adjoint.TraceModel):
the transposed step against the forward step by the dot-product identity
<M u, mu> = <u, M^T mu> for every field path, PEC and Mur;
the gradient on PEC, Mur and CPML grids the gradient of a quadratic
trace misfit with respect to the charge table against exact central
differences of the FP64 oracle (exact because the loss is quadratic in q),
against central differences of the GPU forward at h = 1e-3 relative, and
through torch autograd; argument checks."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

DX = 0.02
DT = W.courant_dt(DX, W.EPS_R_ICE)
Z = 376.730313668 / np.sqrt(W.EPS_R_ICE)


@pytest.fixture(scope="module")
def fd():
    import torch
    torch.cuda.set_device(0)
    import paper_1001_5341_gb300 as m
    return m


def _rand_fields(rng, shape):
    return [rng.standard_normal(shape).astype(np.float32) * (1.0 if c < 3 else 1.0 / Z) for c in range(6)]


def _fields(sim):
    return [sim.field(c).astype(np.float64) for c in range(6)]


@pytest.mark.parametrize("boundary", ["pec", "mur", "cpml"])
@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("n", [1, 7])
def test_transposed_step_dot_product(fd, kernel, n, boundary):
    """Random fields with zero CPML memory in both u and mu: the identity
    then holds on the fields, and over n > 1 steps it covers the memory's
    whole evolution inside M^n and (M^T)^n."""
    nx, ny, nz = 40, 36, 50
    bd = {"pec": fd.FDTD_PEC, "mur": fd.FDTD_MUR1, "cpml": fd.FDTD_CPML}[boundary]
    npml = 6 if boundary == "cpml" else 0
    rng = np.random.default_rng(10 + kernel + n)
    a = fd.Simulation(nx, ny, nz, DX, DT, W.EPS_R_ICE, boundary=bd, npml=npml)
    b = fd.Simulation(nx, ny, nz, DX, DT, W.EPS_R_ICE, boundary=bd, npml=npml)
    for s in (a, b):
        s.set_kernel(kernel)
    u = _rand_fields(rng, a.shape)
    mu = _rand_fields(rng, a.shape)
    for c in range(6):
        a.set_field(c, u[c])
        b.set_field(c, mu[c])
    u0, mu0 = _fields(a), _fields(b)          # as stored (cells outside the state are zero)
    a.step(n)
    b.adjoint_step(n)
    a.sync()
    b.sync()
    Mu, MTmu = _fields(a), _fields(b)
    lhs = sum(float((x * y).sum()) for x, y in zip(Mu, mu0))
    rhs = sum(float((x * y).sum()) for x, y in zip(u0, MTmu))
    scale = np.sqrt(sum(float((x * x).sum()) for x in Mu)) * np.sqrt(sum(float((y * y).sum()) for y in mu0))
    assert abs(lhs - rhs) <= 1e-5 * scale, (lhs, rhs, scale)
    # the transpose is not the step itself
    assert np.abs(np.concatenate([x.ravel() for x in MTmu]) - np.concatenate([x.ravel() for x in _fields_after(fd, mu, kernel, n, bd, npml)])).max() > 0


def _fields_after(fd, f, kernel, n, bd, npml):
    s = fd.Simulation(40, 36, 50, DX, DT, W.EPS_R_ICE, boundary=bd, npml=npml)
    s.set_kernel(kernel)
    for c in range(6):
        s.set_field(c, f[c])
    s.step(n)
    return _fields(s)


def _problem(nbins=24, boundary=None):
    nx, ny, nz = (40, 40, 64) if boundary == "cpml" else (24, 24, 48)
    steps = 100
    z0, bin_dz = 0.06, 0.05
    zb = z0 + bin_dz * np.arange(nbins)
    q = -1e-9 * np.exp(-0.5 * ((zb - 0.5) / 0.2) ** 2) * (1 + 0.3 * np.sin(7 * zb))
    L = 1
    w = np.exp(-0.5 * (np.arange(-L, L + 1)[:, None] ** 2 + np.arange(-L, L + 1)[None, :] ** 2))
    w = (w / w.sum()).ravel()
    cx, cy = nx // 2 * DX, ny // 2 * DX
    xyz = np.array([[cx + 0.10, cy, 0.30], [cx, cy + 0.16, 0.55], [cx - 0.12, cy - 0.08, 0.80],
                    [cx + 0.2, cy + 0.06, 0.42]])
    P = dict(nx=nx, ny=ny, nz=nz, steps=steps, q=q, z0=z0, bin_dz=bin_dz, v=W.C0, w=w, L=L, xyz=xyz, npml=0)
    if boundary is not None:
        P["boundary"] = {"pec": oracle.PEC, "mur": oracle.MUR1, "cpml": oracle.CPML}[boundary]
        P["npml"] = 6 if boundary == "cpml" else 0
    return P


def _oracle_traces(P, q):
    o = oracle.Oracle(P["nx"], P["ny"], P["nz"], DX, DT, W.EPS_R_ICE, boundary=P.get("boundary", oracle.PEC),
                      npml=P["npml"])
    o.set_shower(q, P["z0"], P["bin_dz"], P["v"], P["w"], P["L"])
    o.set_probes(P["xyz"], P["steps"])
    o.step(P["steps"])
    return o.probes()


def _gpu_sim(fd, P):
    s = fd.Simulation(P["nx"], P["ny"], P["nz"], DX, DT, W.EPS_R_ICE, boundary=P.get("boundary", fd.FDTD_PEC),
                      npml=P["npml"])
    s.set_probes(P["xyz"], P["steps"])
    return s


def _gpu_traces(s, P, q):
    s.reset()
    s.set_shower(q, P["z0"], P["bin_dz"], P["v"], P["w"], P["L"])
    s.step(P["steps"])
    return s.probes().astype(np.float64)


@pytest.mark.parametrize("boundary", ["pec", "mur", "cpml"])
def test_gradient_matches_exact_oracle_differences(fd, boundary):
    import torch
    P = _problem(boundary=boundary)
    q = P["q"]
    target = _oracle_traces(P, q * 0.8 + 2e-11 * np.cos(np.arange(q.size)))
    # L(q) = 1/2 sum (y - target)^2 is quadratic in q: central differences are exact
    def loss(qq):
        return 0.5 * float(((_oracle_traces(P, qq) - target) ** 2).sum())
    h = 1e-3 * np.abs(q).max()
    g_ref = np.array([(loss(q + h * e) - loss(q - h * e)) / (2 * h) for e in np.eye(q.size)])
    s = _gpu_sim(fd, P)
    y = _gpu_traces(s, P, q)
    dl = torch.tensor((y - target).astype(np.float32), device="cuda").contiguous()
    g = s.adjoint_gradient(dl, P["steps"])
    rel = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    assert rel <= 1e-3, rel
    assert s.steps_done == 0


def test_gradient_matches_gpu_central_differences(fd):
    import torch
    P = _problem()
    q = P["q"]
    s = _gpu_sim(fd, P)
    target = _gpu_traces(s, P, q * 1.1)
    y = _gpu_traces(s, P, q)
    dl = torch.tensor((y - target).astype(np.float32), device="cuda").contiguous()
    g = s.adjoint_gradient(dl, P["steps"])
    for b in np.argsort(-np.abs(g))[:4]:
        h = 1e-3 * abs(q[b])
        e = np.zeros_like(q)
        e[b] = h
        lp = 0.5 * ((_gpu_traces(s, P, q + e) - target) ** 2).sum()
        lm = 0.5 * ((_gpu_traces(s, P, q - e) - target) ** 2).sum()
        fdg = (lp - lm) / (2 * h)
        assert abs(fdg - g[b]) <= 2e-2 * abs(g[b]), (b, fdg, g[b])


def test_autograd_function(fd):
    import torch
    from paper_1001_5341_gb300.adjoint import TraceModel
    P = _problem()
    s = _gpu_sim(fd, P)
    m = TraceModel(s, P["z0"], P["bin_dz"], P["v"], P["w"], P["L"], P["steps"])
    target = m(torch.tensor(P["q"] * 0.9)).detach()
    q = torch.tensor(P["q"], requires_grad=True)
    y = m(q)
    loss = 0.5 * ((y.double() - target.double()) ** 2).sum()
    loss.backward()
    dl = (y.detach() - target).float().contiguous()
    direct = s.adjoint_gradient(dl, P["steps"])
    assert np.allclose(q.grad.numpy(), direct, rtol=1e-6, atol=1e-12 * np.abs(direct).max())
    assert np.abs(direct).max() > 0


def test_adjoint_argument_checks(fd):
    import torch
    P = _problem()
    s = _gpu_sim(fd, P)
    dl = torch.zeros((4, P["steps"], 2), dtype=torch.float32, device="cuda")
    with pytest.raises(fd.FdtdError):       # no shower
        fd.check(fd.fdtd_adjoint_gradient(s.h, fd._vp(dl.data_ptr()), P["steps"], fd._vp(dl.data_ptr()), 1))
    s.set_shower(P["q"], P["z0"], P["bin_dz"], P["v"], P["w"], P["L"])
    with pytest.raises(fd.FdtdError):       # more steps than the trace holds
        s.adjoint_gradient(dl, P["steps"] + 1)
    with pytest.raises(ValueError):
        s.adjoint_gradient(dl.double(), P["steps"])
