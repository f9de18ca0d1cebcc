"""Macro-elements of uneven degree p and micro-element count m in one
context (independent elements, as in the uneven batch workload): every
element's residual, b-hat^K and recovered dV^K against the oracle's one-element
problem; the same batch streamed in waves (a small memory budget) against the
resident one; the autotuner's record."""
import numpy as np
import pytest

import oracle
from paper_2507_22195_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# the oracle's dense A_qq limits the viscous elements it can condense to n <= 7
VISCOUS_SPECS = [(1, 2), (2, 2), (3, 2), (1, 3), (2, 3), (1, 4), (2, 2), (1, 2), (3, 1), (2, 1), (3, 2)]
INVISCID_SPECS = [(4, 2), (2, 2), (1, 3), (3, 2), (4, 1), (2, 4), (1, 2), (2, 2)]
_REF = {}


def _case(viscous):
    mesh = I.uneven_batch(0, 22199, specs=VISCOUS_SPECS if viscous else INVISCID_SPECS)
    st = I.make_uneven_state(mesh, 1e-2, 22200, 22201, 22202, viscous=viscous)
    kw = dict(flux=1, Mach=0.1, Re=1600.0, Pr=0.71, viscous=int(viscous))
    dvh = I.random_direction(st.vhat.shape, 82, 1e-3)
    if viscous not in _REF:
        prm = oracle.params(**kw)
        ref = oracle.condense_uneven(prm, mesh, st, range(mesh.nK), dvh, procs=8)
        rv = []
        voff, toff = mesh.voff, mesh.toff
        for K in range(mesh.nK):
            em = mesh.element_mesh(K)
            vh = np.stack([st.vhat[toff[g]:toff[g + 1]] for g in mesh.face_gid[K]])
            q = None if st.q is None else st.q[3 * voff[K]:3 * voff[K + 1]]
            rv.append(oracle.residual_K(prm, em.p, em.m, mesh.boxes[K], st.v[voff[K]:voff[K + 1]],
                                        st.vstar[voff[K]:voff[K + 1]], vh, q)[0])
        _REF[viscous] = (ref, rv)
    return mesh, st, kw, dvh, _REF[viscous]


def _dev(st):
    d = torch.device("cuda:0")
    q = None if st.q is None else torch.tensor(st.q, device=d)
    return torch.tensor(st.v, device=d), torch.tensor(st.vhat, device=d), q, torch.tensor(st.vstar, device=d)


def _errors(mesh, bh, dV, RV, ref, rv):
    voff, toff = mesh.voff, mesh.toff
    e = []
    for K, (bh_o, dV_o, _, _) in enumerate(ref):
        b = np.stack([bh[toff[g]:toff[g + 1]] for g in mesh.face_gid[K]]).reshape(bh_o.shape)
        e.append((np.linalg.norm(b - bh_o) / np.linalg.norm(bh_o),
                  np.linalg.norm(dV[voff[K]:voff[K + 1]] - dV_o.ravel()) / np.linalg.norm(dV_o),
                  np.linalg.norm(RV[voff[K]:voff[K + 1]] - rv[K]) / np.linalg.norm(rv[K])))
    return np.array(e)


@pytest.mark.parametrize("viscous", [True, False])
@pytest.mark.parametrize("prec", [0, 4])
def test_uneven_batch_matches_oracle(viscous, prec):
    from paper_2507_22195_gb300 import mehdg as M
    mesh, st, kw, dvh, (ref, rv) = _case(viscous)
    ctx = M.BatchContext(mesh, prec=prec, **kw)
    ctx.set_state(*_dev(st))
    RV, _, _ = ctx.residual()
    bh = ctx.condense()
    dV = ctx.recover(torch.tensor(dvh, device="cuda:0"))
    torch.cuda.synchronize()
    stat, iters = ctx.status()
    assert (stat == 0).all(), (stat, iters)
    rep = ctx.report()
    assert rep["resident"] and len(rep["groups"]) == len(set(zip(mesh.p, mesh.m)))
    costs = [g["cost_flop"] for g in rep["groups"]]
    assert costs == sorted(costs, reverse=True)
    e = _errors(mesh, bh.cpu().numpy(), dV.cpu().numpy(), RV.cpu().numpy(), ref, rv)
    tol = 1e-10 if prec == 0 else 1e-8
    assert e[:, :2].max() < tol, e
    assert e[:, 2].max() < 1e-11, e
    ctx.close()


def test_uneven_batch_streamed_in_waves_matches_resident(monkeypatch):
    """A memory budget below the batch's size: condense runs every (p, m)
    group in balanced waves of elements and keeps no factors (apply and
    recover report MEHDG_ESTATE); b-hat equals the resident batch's."""
    from paper_2507_22195_gb300 import mehdg as M
    mesh, st, kw, dvh, (ref, rv) = _case(True)
    ctx = M.BatchContext(mesh, prec=4, **kw)
    ctx.set_state(*_dev(st))
    bh_res = ctx.condense().cpu().numpy()
    per = max(g["bytes_per_element"] for g in ctx.report()["groups"])
    ctx.close()
    # one element of the costliest group (p = 3, m = 2, two elements) per wave
    monkeypatch.setenv("MEHDG_BATCH_BUDGET_MB", str(1.05 * per / 1048576.0))
    ctx = M.BatchContext(mesh, prec=4, **kw)
    rep = ctx.report()
    assert not rep["resident"] and any(g["wave"] < g["elements"] for g in rep["groups"])
    ctx.set_state(*_dev(st))
    bh = ctx.condense()
    torch.cuda.synchronize()
    stat, _ = ctx.status()
    assert (stat == 0).all()
    assert np.abs(bh.cpu().numpy() - bh_res).max() <= 1e-13 * np.abs(bh_res).max()
    with pytest.raises(M.MehdgError, match="ESTATE"):
        ctx.recover(torch.tensor(dvh, device="cuda:0"))
    ctx.close()


def test_uneven_batch_autotuner_records_its_choices():
    from paper_2507_22195_gb300 import mehdg as M
    mesh, st, kw, dvh, (ref, rv) = _case(False)
    ctx = M.BatchContext(mesh, prec=4, **kw)
    ctx.set_state(*_dev(st))
    ctx.autotune(trial_max=4)
    rep = ctx.report()
    for g in rep["groups"]:
        # leaf CTAs per SM 1, 2, 4, then the solve's CTAs 1, 2, 4, 8 with the better leaf
        assert g["tuned"] and g["leaf_ctas"] in (1, 2, 4) and g["solve_ctas"] in (0, 1, 2, 4, 8)
        assert len(g["trials"]) == 7 and all(t["ms"] > 0 for t in g["trials"])
        assert min(t["ms"] for t in g["trials"]) == pytest.approx(g["best_ms"] if "best_ms" in g else
                                                                  min(t["ms"] for t in g["trials"]))
    bh = ctx.condense()
    dV = ctx.recover(torch.tensor(dvh, device="cuda:0"))
    torch.cuda.synchronize()
    RV, _, _ = ctx.residual()
    e = _errors(mesh, bh.cpu().numpy(), dV.cpu().numpy(), RV.cpu().numpy(), ref, rv)
    assert e[:, :2].max() < 1e-8, e
    ctx.close()
