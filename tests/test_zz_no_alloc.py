"""The allocation-free residual entry point (mehdg_residual_static).

It serves callers that must not allocate device memory after start-up (a
host application whose own pool allocator owns the GPU, a real-time loop).
Checked through the C-ABI against mehdg_residual, the context-based entry
point, on two calls in a row (the static scratch keeps the previous call's
contents, so the second call shows that everything used is re-initialised).
This file is collected last so that a run that stops at the first failure
has already run every other test.
"""
import numpy as np
import pytest

from paper_2507_22195_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("case", ["vortex_p2m2", "tgv_p3m3"])
def test_static_residual_matches_context_residual(case):
    from paper_2507_22195_gb300 import mehdg as M
    if case == "vortex_p2m2":
        mesh = I.periodic_mesh(2, 2, 2, 0.0, 10.0)
        st = I.make_state(mesh, "vortex", 1e-3, 22195, 22196, period=10.0)
    else:
        mesh = I.periodic_mesh((2, 2, 1), 3, 3)
        st = I.make_state(mesh, "tgv", 1e-3, 22197, 22198, M0=0.1)
    dev = torch.device("cuda:0")
    v, vh, vs = (torch.tensor(a, device=dev) for a in (st.v, st.vhat, st.vstar))
    ctx = M.Context(mesh, flux=M.MEHDG_FLUX_KEPES, prec=M.MEHDG_FP64, Mach=0.1)
    ctx.set_state(v, vh, None, vs)
    RV_ref, _, RH_ref = ctx.residual()
    torch.cuda.synchronize()
    prm = M.mehdg_default_params(flux=M.MEHDG_FLUX_KEPES, Mach=0.1)
    box = torch.tensor(mesh.boxes, device=dev)
    gid = torch.tensor(mesh.face_gid, device=dev)
    for call in range(2):
        RV = torch.full_like(RV_ref, np.nan)
        RH = torch.full_like(RH_ref, np.nan)
        M.mehdg_residual_static(prm, mesh.p, mesh.m, box, gid, mesh.n_global_faces, v, vh, None, vs, RV, None, RH)
        torch.cuda.synchronize()
        assert rel(RV, RV_ref) < 1e-11, (call, rel(RV, RV_ref))
        assert rel(RH, RH_ref) < 1e-11, (call, rel(RH, RH_ref))
    ctx.close()


def test_static_residual_rejects_oversized_problems():
    from paper_2507_22195_gb300 import mehdg as M
    dev = torch.device("cuda:0")
    nK, p, m = 400, 4, 4            # 400 x 30 x 17^2 doubles = 27.7 MB > 24 MiB
    box = torch.zeros((nK, 6), dtype=torch.float64, device=dev)
    box[:, 3:] = 1.0
    gid = torch.arange(6 * nK, dtype=torch.int64, device=dev).reshape(nK, 6)
    x = torch.zeros(8, dtype=torch.float64, device=dev)
    prm = M.mehdg_default_params()
    with pytest.raises(M.MehdgError, match="EINVAL"):
        M.mehdg_residual_static(prm, p, m, box, gid, 6 * nK, x, x, None, x, x, None, x)


def test_static_residual_reports_nonphysical_state():
    """beta = -v5 < 0 in one element: MEHDG_ENONPHYS, and the next call on a
    physical state (the status words in the shared array start from zero
    again) returns OK with the context residual's values"""
    from paper_2507_22195_gb300 import mehdg as M
    mesh = I.periodic_mesh(2, 2, 1, 0.0, 10.0)
    st = I.make_state(mesh, "vortex", 1e-3, 22195, 22196, period=10.0)
    dev = torch.device("cuda:0")
    v, vh, vs = (torch.tensor(a, device=dev) for a in (st.v, st.vhat, st.vstar))
    bad = v.clone()
    bad[3, 4, :] = 0.5
    prm = M.mehdg_default_params(flux=M.MEHDG_FLUX_ES, Mach=0.1)
    box = torch.tensor(mesh.boxes, device=dev)
    gid = torch.tensor(mesh.face_gid, device=dev)
    RV = torch.empty((mesh.nK, 5, mesh.Nn), dtype=torch.float64, device=dev)
    RH = torch.empty((mesh.n_global_faces, 5, mesh.n2), dtype=torch.float64, device=dev)
    with pytest.raises(M.MehdgError, match="ENONPHYS"):
        M.mehdg_residual_static(prm, mesh.p, mesh.m, box, gid, mesh.n_global_faces, bad, vh, None, vs, RV, None, RH)
    M.mehdg_residual_static(prm, mesh.p, mesh.m, box, gid, mesh.n_global_faces, v, vh, None, vs, RV, None, RH)
    ctx = M.Context(mesh, flux=M.MEHDG_FLUX_ES, prec=M.MEHDG_FP64, Mach=0.1)
    ctx.set_state(v, vh, None, vs)
    RV_ref, _, RH_ref = ctx.residual()
    torch.cuda.synchronize()
    assert rel(RV, RV_ref) < 1e-11 and rel(RH, RH_ref) < 1e-11
    ctx.close()
