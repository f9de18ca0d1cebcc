"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle, on the
same seeded inputs, element by element.

Errors are relative 2-norms taken per element (per global face for trace
arrays) and maximised over the elements, together with the relative 2-norm
of the whole array; the larger of the two must be below:
  residual R_V, R_Q, R_Vhat (FP64 kernels)                    1e-11
  condensed b-hat, recovered dV, dQ, A-hat x, FP64 LU         1e-10
  same with the mixed-precision LU after FP64 refinement      1e-8
"""
import numpy as np
import pytest

import oracle
from paper_2507_22195_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FLUX = {0: "EC", 1: "ES", 2: "KEPES"}


def M():
    from paper_2507_22195_gb300 import mehdg
    return mehdg


def rel(a, b):
    """max over the leading index (element or global face) of
    ||a_i - b_i|| / ||b_i||, and the whole array's relative error; blocks
    whose norm is below 1e-6 of the largest block are measured against that
    floor (an exactly vanishing block would otherwise divide by zero)"""
    a = a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
    b = np.asarray(b)
    a2, b2 = a.reshape(a.shape[0], -1), b.reshape(b.shape[0], -1)
    nb = np.linalg.norm(b2, axis=1)
    floor = max(1e-6 * nb.max(), 1e-300)
    per = np.linalg.norm(a2 - b2, axis=1) / np.maximum(nb, floor)
    glob = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
    return float(max(per.max(), glob))


def to_dev(st):
    d = torch.device("cuda:0")
    q = None if st.q is None else torch.tensor(st.q, device=d)
    return (torch.tensor(st.v, device=d), torch.tensor(st.vhat, device=d), q,
            torch.tensor(st.vstar, device=d))


def case(name):
    if name == "vortex_p2m2":
        mesh = I.periodic_mesh(2, 2, 2, 0.0, 10.0)
        st = I.make_state(mesh, "vortex", 1e-3, 22195, 22196, period=10.0)
        return mesh, st, dict(Mach=0.1)
    if name == "vortex_p2m1":
        mesh = I.periodic_mesh(2, 2, 1, 0.0, 10.0)
        st = I.make_state(mesh, "vortex", 1e-3, 22195, 22196, period=10.0)
        return mesh, st, dict(Mach=0.1)
    if name == "tgv_p3m2":
        mesh = I.periodic_mesh((2, 1, 1), 3, 2)
        st = I.make_state(mesh, "tgv", 1e-3, 22197, 22198, M0=0.1)
        return mesh, st, dict(Mach=0.1)
    if name == "tgv_p3m3":
        mesh = I.periodic_mesh((2, 2, 1), 3, 3)
        st = I.make_state(mesh, "tgv", 1e-3, 22197, 22198, M0=0.1)
        return mesh, st, dict(Mach=0.1)
    if name == "tgv_p1m1":
        mesh = I.periodic_mesh(3, 1, 1)
        st = I.make_state(mesh, "tgv", 1e-2, 5, 6, M0=0.3)
        return mesh, st, dict(Mach=0.3)
    if name == "tgv_p4m1":
        mesh = I.periodic_mesh(2, 4, 1)
        st = I.make_state(mesh, "tgv", 1e-2, 5, 6, M0=0.3)
        return mesh, st, dict(Mach=0.3)
    raise ValueError(name)


@pytest.mark.parametrize("name", ["vortex_p2m2", "tgv_p3m3", "tgv_p1m1", "tgv_p4m1"])
@pytest.mark.parametrize("flux", [0, 1, 2])
@pytest.mark.parametrize("time_term", [1, 0])
def test_residual_matches_oracle(name, flux, time_term):
    mesh, st, kw = case(name)
    ctx = M().Context(mesh, flux=flux, prec=M().MEHDG_FP64, time_term=time_term, **kw)
    ctx.set_state(*to_dev(st))
    RV, _, RH = ctx.residual()
    torch.cuda.synchronize()
    stat, _ = ctx.status()
    assert (stat == 0).all()
    prm = oracle.params(flux=flux, time_term=time_term, **kw)
    rv, _, rh = oracle.residual_mesh(prm, mesh, st)
    assert rel(RV, rv) < 1e-11, rel(RV, rv)
    assert rel(RH, rh) < 1e-11, rel(RH, rh)
    ctx.close()


_ORACLE_CACHE = {}


def _oracle_condensed(prm, mesh, st, dvh, key=None):
    """b-hat, the assembled sum of A-hat^K, dV and dQ from the oracle (cached
    per case across the precisions of one test)"""
    if key is not None and key in _ORACLE_CACHE:
        return _ORACLE_CACHE[key]
    bh, Ahats = oracle.condense_mesh(prm, mesh, st, want_Ahat=True)
    A = oracle.assemble_Ahat(mesh, Ahats)
    dV, dQ = oracle.recover_mesh(prm, mesh, st, dvh)
    out = (bh, A, dV, dQ)
    if key is not None:
        _ORACLE_CACHE[key] = out
    return out


CONDENSE_CASES = [(nm, 2, pr) for nm in ("vortex_p2m1", "vortex_p2m2", "tgv_p3m2") for pr in (0, 1, 2, 3, 4)]
# the other fluxes of the vortex workload (EC, ES) and of the inviscid TGV workload (EC)
CONDENSE_CASES += [(nm, fl, pr) for nm, fl in (("vortex_p2m2", 0), ("vortex_p2m2", 1), ("tgv_p3m2", 0))
                   for pr in (0, 3, 4)]


@pytest.mark.parametrize("name,flux,prec", CONDENSE_CASES)
def test_condense_apply_recover_match_oracle(name, flux, prec):
    mesh, st, kw = case(name)
    # the BF16 factors contract the refinement error more slowly: more sweeps
    ctx = M().Context(mesh, flux=flux, prec=prec, refine_max_iter=40 if prec == 2 else 10, **kw)
    v, vh, q, vs = to_dev(st)
    ctx.set_state(v, vh, q, vs)
    bh = ctx.condense()
    dvh_np = I.random_direction(st.vhat.shape, 77, 1e-3)
    dvh = torch.tensor(dvh_np, device="cuda:0")
    y = ctx.apply(dvh)
    dV = ctx.recover(dvh)
    torch.cuda.synchronize()
    stat, iters = ctx.status()
    assert (stat == 0).all(), (stat, iters)
    prm = oracle.params(flux=flux, **kw)
    bh_o, A_o, dV_o, _ = _oracle_condensed(prm, mesh, st, dvh_np, key=("inv", name, flux))
    y_o = (A_o @ dvh_np.ravel()).reshape(dvh_np.shape)
    tol = 1e-10 if prec == 0 else 1e-8
    e = (rel(bh, bh_o), rel(y, y_o), rel(dV, dV_o))
    assert max(e) < tol, (e, iters)
    ctx.close()


@pytest.mark.parametrize("viscous", [False, True])
@pytest.mark.parametrize("prec", [0, 4])
def test_condense_64_elements_matches_oracle(viscous, prec):
    """a 4^3 mesh: every kernel's grid spans 64 elements (more CTAs than the
    small parity cases, grid rows past the first wave of SMs)"""
    mesh = I.periodic_mesh(4, 2, 1)
    st = I.make_state(mesh, "tgv", 1e-2, 5, 6, viscous=viscous, M0=0.3)
    kw = dict(Mach=0.3, Re=100.0, viscous=1) if viscous else dict(Mach=0.3)
    ctx = M().Context(mesh, flux=1, prec=prec, **kw)
    ctx.set_state(*to_dev(st))
    bh = ctx.condense()
    dvh_np = I.random_direction(st.vhat.shape, 79, 1e-3)
    dV = ctx.recover(torch.tensor(dvh_np, device="cuda:0"))
    torch.cuda.synchronize()
    stat, iters = ctx.status()
    assert (stat == 0).all(), (stat, iters)
    prm = oracle.params(flux=1, **kw)
    bh_o, _ = oracle.condense_mesh(prm, mesh, st)
    dV_o, _ = oracle.recover_mesh(prm, mesh, st, dvh_np)
    tol = 1e-10 if prec == 0 else 1e-8
    e = (rel(bh, bh_o), rel(dV, dV_o))
    assert max(e) < tol, (e, iters)
    ctx.close()


# ---------------------------------------------------------------- the bench's LU configuration
BENCH_NK = 160                       # more elements than the GPU's 152 SMs
BENCH_SAMPLE = [0, 77, 151, 159]     # first wave, middle, last of the first wave, second wave


@pytest.fixture(scope="module")
def bench_lu_case():
    """160 elements of the 8^3 x 3^3, p = 3 inviscid TGV (Mach 0.1, KEPES)
    with unshared faces, the state of the benchmark's workload (amplitude
    1e-3, seeds 22197/22198), a seeded trace increment, and the oracle's
    b-hat^K and dV^K for the sample elements (condensed in parallel)."""
    mesh = I.unshared(I.periodic_mesh(8, 3, 3), range(BENCH_NK))
    st = I.make_state(mesh, "tgv", 1e-3, 22197, 22198, M0=0.1)
    dvh = I.random_direction(st.vhat.shape, 80, 1e-3)
    prm = oracle.params(flux=2, Mach=0.1)
    ref = oracle.condense_elements(prm, mesh, st, BENCH_SAMPLE, dvh, procs=len(BENCH_SAMPLE))
    return mesh, st, dvh, ref


@pytest.mark.parametrize("prec,leaf", [(4, 0), (3, 0), (4, 4)])
def test_condense_at_bench_lu_configuration_matches_oracle(bench_lu_case, prec, leaf, monkeypatch):
    """p = 3, m = 3 (N_v = 5000, ld = 5120) with more elements than SMs: the
    LU runs the leaf variants the benchmark runs (two 512-thread CTAs per SM,
    4-, 8- and 32-column sub-panels; with leaf = 4 also the four 256-thread
    CTAs per SM that the leaves of at most 1504 rows take with more than two
    elements per SM) and the one-CTA-per-element solve.  b-hat^K (its faces
    are unshared, so the global b-hat on them is b-hat^K) and the recovered
    dV^K are compared element by element."""
    if leaf:
        monkeypatch.setenv("MEHDG_LEAF_CTAS_PER_SM", str(leaf))
    mesh, st, dvh_np, ref = bench_lu_case
    ctx = M().Context(mesh, flux=2, prec=prec, Mach=0.1)
    ctx.set_state(*to_dev(st))
    bh = ctx.condense()
    dV = ctx.recover(torch.tensor(dvh_np, device="cuda:0"))
    torch.cuda.synchronize()
    stat, iters = ctx.status()
    assert (stat == 0).all(), (np.unique(stat), np.unique(iters))
    bh = bh.cpu().numpy()
    dV = dV.cpu().numpy()
    errs = []
    for K, (bh_o, dV_o, _, _) in zip(BENCH_SAMPLE, ref):
        e_b = np.linalg.norm(bh[6 * K:6 * K + 6] - bh_o) / np.linalg.norm(bh_o)
        e_v = np.linalg.norm(dV[K] - dV_o) / np.linalg.norm(dV_o)
        errs.append((K, e_b, e_v))
    assert max(max(e[1], e[2]) for e in errs) < 1e-8, errs
    ctx.close()


@pytest.mark.parametrize("pairs", [1, 0])
@pytest.mark.parametrize("name", ["vortex_p2m2", "tgv_p3m2"])
def test_lu_pair_and_one_panel_forms_match_oracle(name, pairs, monkeypatch):
    """split BF16 merges the outer updates of two panels into one of depth 512
    (MEHDG_LU_PAIRS=0 selects one update per panel): 3 outer panels (one pair
    and a single panel) and 7 (three pairs and a single panel) per element"""
    monkeypatch.setenv("MEHDG_LU_PAIRS", str(pairs))
    mesh, st, kw = case(name)
    ctx = M().Context(mesh, flux=2, prec=M().MEHDG_MIXED_BF16X3, **kw)
    ctx.set_state(*to_dev(st))
    bh = ctx.condense()
    dvh_np = I.random_direction(st.vhat.shape, 78, 1e-3)
    dV = ctx.recover(torch.tensor(dvh_np, device="cuda:0"))
    torch.cuda.synchronize()
    stat, iters = ctx.status()
    assert (stat == 0).all(), (stat, iters)
    prm = oracle.params(flux=2, **kw)
    bh_o, _ = oracle.condense_mesh(prm, mesh, st)
    dV_o, _ = oracle.recover_mesh(prm, mesh, st, dvh_np)
    e = (rel(bh, bh_o), rel(dV, dV_o))
    assert max(e) < 1e-8, (e, iters)
    ctx.close()


@pytest.mark.parametrize("ctas", [1, 2, 4, 8])
def test_solve_cluster_sizes_match_oracle(ctas, monkeypatch):
    """the solve with 1, 2, 4 and 8 CTAs per element (normally chosen from the
    element count) on a mesh with three outer panels per element"""
    monkeypatch.setenv("MEHDG_SOLVE_CTAS", str(ctas))
    mesh, st, kw = case("vortex_p2m2")
    ctx = M().Context(mesh, flux=2, prec=M().MEHDG_MIXED_BF16X3, **kw)
    v, vh, q, vs = to_dev(st)
    ctx.set_state(v, vh, q, vs)
    bh = ctx.condense()
    dvh_np = I.random_direction(st.vhat.shape, 77, 1e-3)
    dV = ctx.recover(torch.tensor(dvh_np, device="cuda:0"))
    torch.cuda.synchronize()
    stat, iters = ctx.status()
    assert (stat == 0).all(), (stat, iters)
    prm = oracle.params(flux=2, **kw)
    bh_o, _ = oracle.condense_mesh(prm, mesh, st)
    dV_o, _ = oracle.recover_mesh(prm, mesh, st, dvh_np)
    e = (rel(bh, bh_o), rel(dV, dV_o))
    assert max(e) < 1e-8, (e, iters)
    ctx.close()


def test_newton_step_matches_brute_force():
    """condense -> dense global solve of sum A-hat (built column by column with
    apply_condensed) -> recover equals the oracle's monolithic solve"""
    mesh = I.periodic_mesh(2, 1, 1)
    st = I.make_state(mesh, "tgv", 1e-2, 5, 6, M0=0.3)
    ctx = M().Context(mesh, flux=2, prec=M().MEHDG_FP64, Mach=0.3)
    ctx.set_state(*to_dev(st))
    bh = ctx.condense()
    G = st.vhat.size
    A = np.zeros((G, G))
    for j in range(G):
        e = torch.zeros(st.vhat.shape, dtype=torch.float64, device="cuda:0")
        e.view(-1)[j] = 1.0
        A[:, j] = ctx.apply(e).cpu().numpy().ravel()
    x = np.linalg.solve(A, bh.cpu().numpy().ravel()).reshape(st.vhat.shape)
    dV = ctx.recover(torch.tensor(x, device="cuda:0"))
    prm = oracle.params(flux=2, Mach=0.3)
    _, dV_o, dH_o = oracle.brute_force(prm, mesh, st)
    assert rel(x, dH_o) < 1e-9 and rel(dV, dV_o) < 1e-9
    ctx.close()


@pytest.mark.parametrize("prec", [0, 4])
def test_newton_step_with_gmres_trace_solve_matches_brute_force(prec):
    """condense -> GMRES on sum A-hat (matrix-free) -> recover equals the
    oracle's monolithic solve of the whole (V, V-hat) Newton system.  The
    restart length covers the whole trace system of this mesh, so GMRES is
    exact in exact arithmetic (without a preconditioner restarted GMRES
    stagnates on these systems: condition numbers ~1e5, spectrum spread over
    the left half-plane)."""
    mesh = I.periodic_mesh(2, 1, 1)
    st = I.make_state(mesh, "tgv", 1e-2, 5, 6, M0=0.3)
    ctx = M().Context(mesh, flux=2, prec=prec, Mach=0.3)
    ctx.set_state(*to_dev(st))
    bh = ctx.condense()
    x, it, res = ctx.solve_condensed(bh, rtol=1e-13, restart=bh.numel(), max_iter=2 * bh.numel())
    dV = ctx.recover(x)
    torch.cuda.synchronize()
    stat, _ = ctx.status()
    assert (stat == 0).all()
    assert res <= 1e-13 and 0 < it <= bh.numel()
    prm = oracle.params(flux=2, Mach=0.3)
    _, dV_o, dH_o = oracle.brute_force(prm, mesh, st)
    tol = 1e-9 if prec == 0 else 1e-8
    assert rel(x, dH_o) < tol and rel(dV, dV_o) < tol, (rel(x, dH_o), rel(dV, dV_o), it)
    ctx.close()


def test_gmres_reports_no_convergence():
    mesh = I.periodic_mesh(2, 1, 1)
    st = I.make_state(mesh, "tgv", 1e-2, 5, 6, M0=0.3)
    ctx = M().Context(mesh, flux=2, prec=M().MEHDG_FP64, Mach=0.3)
    ctx.set_state(*to_dev(st))
    bh = ctx.condense()
    x = torch.zeros_like(bh)
    it, res = M().mehdg_solve_condensed(ctx.ctx, bh, x, rtol=1e-14, restart=2, max_iter=3, check=False)
    assert it == 3 and res > 1e-14
    with pytest.raises(M().MehdgError):
        M().mehdg_solve_condensed(ctx.ctx, bh, torch.zeros_like(bh), rtol=1e-14, restart=2, max_iter=3)
    ctx.close()


def test_nonphysical_state_reports_status():
    mesh, st, kw = case("vortex_p2m1")
    st.v[3, 4, :] = 0.5           # beta = -v5 < 0 in element 3
    ctx = M().Context(mesh, flux=2, prec=M().MEHDG_FP64, **kw)
    ctx.set_state(*to_dev(st))
    ctx.residual()
    stat, _ = ctx.status()
    assert stat[3] == -2 and (np.delete(stat, 3) == 0).all()
    # the same words through the device form, on the current stream
    d = torch.full((mesh.nK,), 7, dtype=torch.int32, device="cuda:0")
    M().mehdg_status_device(ctx.ctx, d)
    torch.cuda.current_stream().synchronize()
    assert (d.cpu().numpy() == stat).all()
    ctx.close()


def test_bad_arguments_return_einval():
    mesh, st, kw = case("vortex_p2m1")
    with pytest.raises(M().MehdgError, match="EINVAL"):
        ctx = M().Context(mesh, flux=7)
    ctx = M().Context(mesh, **kw)
    with pytest.raises(M().MehdgError, match="ESTATE"):
        ctx.recover(torch.zeros(st.vhat.shape, dtype=torch.float64, device="cuda:0"))
    gid = mesh.face_gid.copy()
    gid[0, 0] = mesh.n_global_faces + 5
    with pytest.raises(M().MehdgError, match="EINVAL"):
        M().mehdg_set_mesh(ctx.ctx, np.full(mesh.nK, 2), np.full(mesh.nK, 1), mesh.boxes, gid,
                           mesh.n_global_faces)
    ctx.close()


# ---------------------------------------------------------------- viscous
def vcase(name):
    p, m = {"p2m1": (2, 1), "p2m2": (2, 2), "p3m1": (3, 1), "p1m2": (1, 2), "p3m2": (3, 2), "p1m4": (1, 4),
            "p3m4": (3, 4)}[name]
    mesh = I.periodic_mesh((2, 1, 1), p, m)
    st = I.make_state(mesh, "tgv", 1e-2, 5, 6, viscous=True, M0=0.3)
    return mesh, st, dict(Mach=0.3, Re=100.0, viscous=1)


@pytest.mark.parametrize("name", ["p2m1", "p2m2", "p3m1", "p3m4"])
@pytest.mark.parametrize("flux", [1, 2])
def test_viscous_residual_matches_oracle(name, flux):
    """p3m4 is the element of the viscous TGV workload (n = 13, N_v = 10985)"""
    mesh, st, kw = vcase(name)
    ctx = M().Context(mesh, flux=flux, prec=M().MEHDG_FP64, **kw)
    ctx.set_state(*to_dev(st))
    RV, RQ, RH = ctx.residual()
    torch.cuda.synchronize()
    prm = oracle.params(flux=flux, **kw)
    rv, rq, rh = oracle.residual_mesh(prm, mesh, st)
    for a, b in ((RV, rv), (RQ, rq), (RH, rh)):
        assert rel(a, b) < 1e-11, rel(a, b)
    ctx.close()


@pytest.mark.parametrize("name", ["p2m1", "p2m2", "p3m1", "p1m2", "p3m2", "p1m4"])
@pytest.mark.parametrize("prec", [0, 3, 4])
def test_viscous_condense_apply_recover_match_oracle(name, prec):
    """Q-elimination (eqs. R2, R3, R5, R6) against the oracle's literal blocks"""
    mesh, st, kw = vcase(name)
    ctx = M().Context(mesh, flux=1, prec=prec, **kw)
    ctx.set_state(*to_dev(st))
    bh = ctx.condense()
    dvh_np = I.random_direction(st.vhat.shape, 78, 1e-3)
    dvh = torch.tensor(dvh_np, device="cuda:0")
    y = ctx.apply(dvh)
    dV, dQ = ctx.recover(dvh, with_dQ=True)
    torch.cuda.synchronize()
    stat, iters = ctx.status()
    assert (stat == 0).all(), (stat, iters)
    prm = oracle.params(flux=1, **kw)
    bh_o, A_o, dV_o, dQ_o = _oracle_condensed(prm, mesh, st, dvh_np, key=("vis", name))
    y_o = (A_o @ dvh_np.ravel()).reshape(dvh_np.shape)
    tol = 1e-10 if prec == 0 else 1e-8
    e = (rel(bh, bh_o), rel(y, y_o), rel(dV, dV_o), rel(dQ, dQ_o))
    assert max(e) < tol, (e, iters)
    ctx.close()


@pytest.mark.parametrize("prec", [4, 3])
def test_viscous_p3m4_mixed_matches_fp64(prec):
    """The element of the viscous TGV workload (p = 3, m = 4: N_v = 10985,
    N_q = 32955).  The oracle's literal blocks are out of reach at this size
    (its dense A_qq alone is 8.7 GB per element, and its GEPP takes hours), so
    the mixed-precision condensation is compared with the FP64 GPU path, whose
    residual at this size and whose condensation at p3m2 and p1m4 are checked
    against the oracle above."""
    mesh, st, kw = vcase("p3m4")
    dvh_np = I.random_direction(st.vhat.shape, 81, 1e-3)
    out = {}
    for pr in (0, prec):
        ctx = M().Context(mesh, flux=1, prec=pr, **kw)
        ctx.set_state(*to_dev(st))
        bh = ctx.condense()
        dV, dQ = ctx.recover(torch.tensor(dvh_np, device="cuda:0"), with_dQ=True)
        torch.cuda.synchronize()
        stat, iters = ctx.status()
        assert (stat == 0).all(), (pr, stat, iters)
        out[pr] = (bh.cpu().numpy(), dV.cpu().numpy(), dQ.cpu().numpy())
        ctx.close()
    e = [rel(a, b) for a, b in zip(out[prec], out[0])]
    assert max(e) < 1e-8, e
