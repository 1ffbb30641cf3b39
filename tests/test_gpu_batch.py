"""Batched ensemble: instances of uneven size through persistent grids and a
CUDA graph.  The three execution modes give bitwise identical results for a
given brick shape; every instance matches the oracle; autotuning keeps parity."""
import numpy as np
import pytest

import parity

from paper_2601_08266_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


@pytest.fixture(scope="module")
def fsi():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2601_08266_gb300 as pkg
    return pkg


def T(a, dtype):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda").to(dtype).contiguous()


def H(t):
    return t.detach().cpu().numpy().astype(np.float64)


def rel(a, b, grid=None):
    """Worst local relative error of a against b: momentum and continuity
    rows, boundary and interior nodes (when grid is given) apart, norm-wise
    and largest entry (tests/parity.py)."""
    return parity.rel_local(np.asarray(a), b, grid)


def rel_norm(a, b):
    """Norm-wise distance of a whole solution vector from a reference one."""
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a) - b) / (nb if nb > 0 else 1.0)


SHAPES = [((5, 5, 5), None, 300), ((9, 7, 11), (0.11, 0.14, 0.09), 800), ((12, 12, 12), None, 0),
          ((3, 4, 2), (0.3, 0.25, 0.5), 50), ((16, 8, 6), None, 2000), ((7, 13, 4), None, 400)]


def build(fsi, prec, stream):
    import torch
    dt = torch.float64 if prec == "f64" else torch.float32
    P = fsi.FSI_F64 if prec == "f64" else fsi.FSI_F32
    rng = np.random.default_rng(42)
    meshes, items, host = [], [], []
    for i, (N, h, m) in enumerate(SHAPES):
        mu = float(np.exp(rng.uniform(np.log(1e-3), np.log(1e-1))))
        mesh = fsi.Mesh(N, h=h, rho=1.0, mu=mu, dt=1e-3, rho_inf=0.5, device=0, stream=stream)
        n = mesh.n_nodes
        U = rng.uniform(-1, 1, (n, 4))
        A = rng.uniform(-1, 1, (n, 4))
        A[:, 3] = 1.0
        x = rng.uniform(-1, 1, (n, 4))
        if prec == "f32":
            U, A, x = (a.astype(np.float32).astype(np.float64) for a in (U, A, x))
        it = dict(U=T(U, dt), A=T(A, dt), x=T(x, dt),
                  R=torch.zeros((n, 4), dtype=dt, device="cuda"),
                  Jx=torch.zeros((n, 4), dtype=dt, device="cuda"),
                  F=torch.zeros((n, 4), dtype=dt, device="cuda"),
                  cell_start=torch.empty(mesh.n_elems + 1, dtype=torch.int32, device="cuda"))
        ext = np.asarray(mesh.h) * np.asarray(N)
        X = rng.uniform(0, 1, (m, 3)) * ext
        lam = rng.normal(size=(m, 3))
        if prec == "f32":
            lam = lam.astype(np.float32).astype(np.float64)
        elem = torch.empty(m, dtype=torch.int32, device="cuda")
        xi = torch.empty((m, 3), dtype=torch.float64, device="cuda")
        perm = torch.empty(m, dtype=torch.int32, device="cuda")
        with torch.cuda.stream(stream_obj(stream)):
            fsi.fsi_locate(mesh, T(X, torch.float64), elem, xi, it["cell_start"], perm)
        it.update(elem=elem, xi=xi.to(dt).contiguous(), perm=perm, lam=T(lam, dt),
                  u=torch.zeros((m, 3), dtype=dt, device="cuda"))
        meshes.append(mesh)
        items.append(it)
        host.append(dict(N=N, h=h, mu=mu, U=U, A=A, x=x, X=X, lam=lam))
    torch.cuda.synchronize()
    return meshes, items, host, P


_streams = {}


def stream_obj(handle):
    return _streams[handle]


def outputs(items):
    return [tuple(H(it[k]) for k in ("R", "Jx", "u", "F")) for it in items]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_batch_modes_agree_and_match_oracle(fsi, oracle, prec):
    import torch
    s = torch.cuda.Stream()
    _streams[s.cuda_stream] = s
    meshes, items, host, P = build(fsi, prec, s.cuda_stream)
    b = fsi.Batch(meshes, items, P, s.cuda_stream)
    res = {}
    for mode in (fsi.FSI_BATCH_PER_INSTANCE, fsi.FSI_BATCH_PERSISTENT, fsi.FSI_BATCH_GRAPH):
        for it in items:
            for k in ("R", "Jx", "u", "F"):
                it[k].fill_(float("nan"))
        b.run(mode)
        s.synchronize()
        res[mode] = outputs(items)
    for mode in (fsi.FSI_BATCH_PERSISTENT, fsi.FSI_BATCH_GRAPH):
        for a, c in zip(res[mode], res[fsi.FSI_BATCH_PER_INSTANCE]):
            for x, y in zip(a, c):
                assert np.array_equal(x[..., :3] if x.shape[-1] == 4 else x,
                                      y[..., :3] if y.shape[-1] == 4 else y)
            assert np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1])
    # every instance against the oracle
    from oracle import timeint
    for (R, Jx, u, F), hst in zip(res[fsi.FSI_BATCH_GRAPH], host):
        g = oracle.core.Grid(hst["N"], h=hst["h"])
        phys = dict(rho=1.0, mu=hst["mu"], dt=1e-3)
        c_a, c_v = timeint.chain_factors(0.5, 1e-3)
        assert rel(R, oracle.core.residual(g, phys, hst["U"], hst["A"]), g.N) < TOL[prec]
        assert rel(Jx, oracle.core.jacobian_apply(g, phys, hst["U"], hst["A"], hst["x"], c_a,
                                                  c_v), g.N) < TOL[prec]
        if len(hst["X"]):
            e, xi, _ = oracle.core.locate(g, hst["X"])
            xiw = xi.astype(np.float32).astype(np.float64) if prec == "f32" else xi
            assert rel(u, oracle.core.interp(g, e, xiw, hst["U"])) < TOL[prec]
            Fo = oracle.core.spread(g, e, xiw, hst["lam"])
            assert rel(F[:, :3], Fo[:, :3], g.N) < TOL[prec]
        else:
            assert np.all(F[:, :3] == 0)
    b.close()


def test_batch_autotune_keeps_parity(fsi, oracle):
    import torch
    s = torch.cuda.Stream()
    _streams[s.cuda_stream] = s
    meshes, items, host, P = build(fsi, "f32", s.cuda_stream)
    b = fsi.Batch(meshes, items, P, s.cuda_stream)
    t = b.autotune(reps=1)
    assert t["n_candidates"] if "n_candidates" in t else len(t["candidates"]) > 0
    assert t["seconds"] > 0 and min(c[4] for c in t["candidates"]) == pytest.approx(t["seconds"])
    b.run(fsi.FSI_BATCH_GRAPH)
    s.synchronize()
    from oracle import timeint
    c_a, c_v = timeint.chain_factors(0.5, 1e-3)
    for it, hst in zip(items, host):
        g = oracle.core.Grid(hst["N"], h=hst["h"])
        phys = dict(rho=1.0, mu=hst["mu"], dt=1e-3)
        assert rel(H(it["Jx"]), oracle.core.jacobian_apply(g, phys, hst["U"], hst["A"], hst["x"],
                                                           c_a, c_v)) < 1e-5
    b.close()


def test_mesh_brick_shapes_keep_parity(fsi, oracle):
    import torch
    N = (11, 9, 13)
    mesh = fsi.Mesh(N, device=0)
    rng = np.random.default_rng(3)
    n = mesh.n_nodes
    U, A, x = (rng.uniform(-1, 1, (n, 4)) for _ in range(3))
    g = oracle.core.Grid(N)
    phys = dict(rho=1.0, mu=0.01, dt=1e-3)
    from oracle import timeint
    c_a, c_v = timeint.chain_factors(0.5, 1e-3)
    ref = oracle.core.jacobian_apply(g, phys, U, A, x, c_a, c_v)
    for bx, by, bz, th in [(4, 4, 4, 64), (16, 4, 2, 256), (2, 2, 2, 32), (8, 8, 4, 128)]:
        fsi.fsi_mesh_set_brick(mesh, 1, fsi.FSI_F64, bx, by, bz, th)
        J = torch.empty((n, 4), dtype=torch.float64, device="cuda")
        fsi.fsi_jacobian_apply(mesh, fsi.FSI_F64, T(U, torch.float64), T(A, torch.float64), None,
                               T(x, torch.float64), J)
        torch.cuda.synchronize()
        assert rel(H(J), ref) < 1e-12, (bx, by, bz, th)
    with pytest.raises(fsi.FsiError):
        fsi.fsi_mesh_set_brick(mesh, 1, fsi.FSI_F64, 32, 32, 4, 256)


@pytest.mark.parametrize("prec", ["df64", "f32"])
def test_mesh_autotune_keeps_parity(fsi, oracle, prec):
    """The single-mesh autotuner times every candidate brick of both operators,
    keeps the fastest, and the tuned kernels still match the oracle."""
    import torch
    N = (14, 9, 11)
    mesh = fsi.Mesh(N, device=0, has_s=True)
    P = fsi.FSI_DF64 if prec == "df64" else fsi.FSI_F32
    dt = torch.float64 if prec == "df64" else torch.float32
    picks = []
    for op in (0, 1):
        t = fsi.fsi_mesh_autotune(mesh, op, P, reps=2)
        assert len(t["candidates"]) == 10 and t["seconds"] > 0
        assert min(c[2] for c in t["candidates"]) == pytest.approx(t["seconds"])
        assert (t["brick"], t["threads"]) in [(c[0], c[1]) for c in t["candidates"]]
        picks.append(t)
    rng = np.random.default_rng(4)
    n = mesh.n_nodes
    U, A, x = (rng.uniform(-1, 1, (n, 4)) for _ in range(3))
    A[:, 3] = rng.uniform(1.0, 3.0, n)
    if prec == "f32":
        U, A, x = (a.astype(np.float32).astype(np.float64) for a in (U, A, x))
    g = oracle.core.Grid(N)
    phys = dict(rho=1.0, mu=0.01, dt=1e-3, has_s=True)
    from oracle import timeint
    c_a, c_v = timeint.chain_factors(0.5, 1e-3)
    R = torch.empty((n, 4), dtype=dt, device="cuda")
    J = torch.empty((n, 4), dtype=dt, device="cuda")
    fsi.fsi_residual(mesh, P, T(U, dt), T(A, dt), None, R)
    fsi.fsi_jacobian_apply(mesh, P, T(U, dt), T(A, dt), None, T(x, dt), J)
    torch.cuda.synchronize()
    tol = 1e-12 if prec == "df64" else 1e-5
    assert rel(H(R), oracle.core.residual(g, phys, U, A)) < tol, picks
    assert rel(H(J), oracle.core.jacobian_apply(g, phys, U, A, x, c_a, c_v)) < tol, picks
    with pytest.raises(fsi.FsiError):
        fsi.fsi_mesh_autotune(mesh, 3, P)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_batch_locates_its_points(fsi, oracle, prec):
    """Items that bring raw points: the batched step (per instance, persistent
    grids and the CUDA graph) locates them and builds every instance's cell
    table itself.  elem, cell_start and perm equal fsi_locate's bit for bit,
    xi equals fsi_locate's (rounded to FP32 in an FP32 batch), and R, Jx, u, F
    equal those of the same batch fed fsi_locate's tables.  The points include
    outside points, points on the far faces and an instance without points."""
    import torch
    s = torch.cuda.Stream()
    _streams[s.cuda_stream] = s
    meshes, items, host, P = build(fsi, prec, s.cuda_stream)
    dt = torch.float64 if prec == "f64" else torch.float32
    ref_tables = []
    loc_items = []
    for i, (mesh, it, hst) in enumerate(zip(meshes, items, host)):
        X = hst["X"]
        if len(X):
            ext = np.asarray(mesh.h) * np.asarray(hst["N"])
            X = np.concatenate([X, inputs.edge_points(hst["N"], seed=len(X), m_random=20)
                                * ext[None, :]])
            X[::7] *= 1.05           # some outside the box
        m = X.shape[0]
        Xd = T(X, torch.float64)
        e = torch.empty(m, dtype=torch.int32, device="cuda")
        xi = torch.empty((m, 3), dtype=torch.float64, device="cuda")
        cs = torch.empty(mesh.n_elems + 1, dtype=torch.int32, device="cuda")
        pm = torch.empty(m, dtype=torch.int32, device="cuda")
        with torch.cuda.stream(s):
            fsi.fsi_locate(mesh, Xd, e, xi, cs, pm)
        s.synchronize()
        ref_tables.append((e.cpu().numpy(), xi.to(dt).cpu().numpy(), cs.cpu().numpy(),
                           pm.cpu().numpy()))
        lam = T(np.random.default_rng(m).normal(size=(m, 3)), dt)
        base = {k: it[k] for k in ("U", "A", "x")}
        fed = dict(base, R=torch.zeros_like(it["R"]), Jx=torch.zeros_like(it["R"]),
                   F=torch.zeros_like(it["F"]), cell_start=cs, elem=e, xi=xi.to(dt).contiguous(),
                   perm=pm, lam=lam, u=torch.zeros((m, 3), dtype=dt, device="cuda"))
        own = dict(base, R=torch.zeros_like(it["R"]), Jx=torch.zeros_like(it["R"]),
                   F=torch.zeros_like(it["F"]),
                   cell_start=torch.full_like(cs, -7) if m else cs.clone(),
                   elem=torch.full_like(e, 9),
                   xi=torch.full((m, 3), 5.0, dtype=dt, device="cuda"),
                   perm=torch.full_like(pm, -3), lam=lam,
                   u=torch.zeros((m, 3), dtype=dt, device="cuda"), X=Xd)
        items[i] = fed
        loc_items.append(own)
    b_fed = fsi.Batch(meshes, items, P, s.cuda_stream)
    b_fed.run(fsi.FSI_BATCH_PERSISTENT)
    s.synchronize()
    want = outputs(items)
    b_own = fsi.Batch(meshes, loc_items, P, s.cuda_stream)
    for mode in (fsi.FSI_BATCH_PER_INSTANCE, fsi.FSI_BATCH_PERSISTENT, fsi.FSI_BATCH_GRAPH):
        for it in loc_items:
            if it["elem"].shape[0]:   # an empty X is NULL: that item keeps its table
                it["cell_start"].fill_(-7)
            it["elem"].fill_(9)
            it["perm"].fill_(-3)
            it["xi"].fill_(5.0)
            for k in ("R", "Jx", "u", "F"):
                it[k].fill_(float("nan"))
        for _ in range(2):           # the second step starts from the first's tables
            b_own.run(mode)
        s.synchronize()
        for it, (e, xi, cs, pm) in zip(loc_items, ref_tables):
            assert np.array_equal(it["elem"].cpu().numpy(), e), mode
            assert np.array_equal(it["cell_start"].cpu().numpy(), cs), mode
            assert np.array_equal(it["perm"].cpu().numpy(), pm), mode
            assert np.array_equal(it["xi"].cpu().numpy(), xi), mode
        for a, c in zip(outputs(loc_items), want):
            for x, y in zip(a, c):
                assert np.array_equal(x[..., :3] if x.shape[-1] == 4 else x,
                                      y[..., :3] if y.shape[-1] == 4 else y), mode
    b_own.close()
    b_fed.close()
