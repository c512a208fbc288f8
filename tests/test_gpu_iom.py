"""Incomplete orthogonalisation (the procedure KIOPS uses in place of Arnoldi,
Sec. 1) on the CUDA path, against the oracle run with the same window.

FP64 form with the oracle's decisions replayed: 1e-11 relative (rounding
order only: the GPU forms the window's inner products in one classical pass,
the oracle sweeps them in modified Gram-Schmidt order; the window vectors are
mutually orthogonal, so both are the same projection).  Mixed and
float-float forms: 1e-6 against the oracle's full-Arnoldi step, the bar of
those forms."""
import numpy as np
import pytest

from oracle import dg, integrators, krylov
from paper_2011_01316_gb300 import inputs
from tests.test_gpu_parity import CASES, MIXED_PRECS, PRECS, TOL_MIXED, TOL_STEP64, _replay_from, rel, state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_01316_gb300 import expdg
    return expdg


def make(E, case, iop, prec=0, scheme=2, tol=1e-10, m_max=64):
    c = CASES[case]
    kw = dict(eq=c["eq"], dim=c["dim"], p=c["p"], ne=list(c["ne"]) + [1] * (3 - c["dim"]),
              lo=list(c["lo"]) + [0.0] * (3 - c["dim"]), hi=list(c["hi"]) + [1.0] * (3 - c["dim"]),
              prec=prec, scheme=scheme, krylov_tol=tol, m_max=m_max, m_step=5, max_substeps=32, gamma=1.4,
              iop=iop)
    ctx = E.Context(**kw)
    mesh = dg.Mesh(dim=c["dim"], p=c["p"], ne=c["ne"], lo=c["lo"], hi=c["hi"],
                   eq="burgers" if c["eq"] == 1 else "euler")
    return ctx, mesh


@pytest.mark.parametrize("iop", [1, 2, 4, 8])
@pytest.mark.parametrize("P", [0, 1, 3])
@pytest.mark.parametrize("case", ["burgers1d_p2", "euler2d_p4", "euler3d_p2"])
def test_phi_iom_replayed(E, case, P, iop):
    rng = np.random.default_rng(60 + P)
    ctx, mesh = make(E, case, iop)
    q = state(mesh, rng).reshape(-1)
    tau = 0.05
    c = [rng.standard_normal(q.size) * 0.1 for _ in range(P + 1)]
    if P > 0:
        c[0] = np.zeros_like(q)
    ref, st = krylov.phi_sum(lambda x: tau * dg.jv(mesh, q, x).reshape(-1), c, tol=1e-10, iop=iop)
    rep = [(0, m, s, e) for (s, m, e) in st.trace]
    got, gst, gtr = ctx.phi(q, tau, [None if (i == 0 and P > 0) else np.ascontiguousarray(ci)
                                     for i, ci in enumerate(c)], replay=rep)
    assert rel(got, ref) <= TOL_STEP64
    assert [(m, s) for (_, m, s, _) in gtr] == [(m, s) for (s, m, _) in st.trace]


@pytest.mark.parametrize("iop", [2, 4])
@pytest.mark.parametrize("case", ["burgers1d_p2", "euler2d_p4", "euler3d_p2"])
def test_phi_iom_adaptive_agrees(E, case, iop):
    """Decisions taken on the GPU agree with the oracle's (same window) to 10 tol."""
    rng = np.random.default_rng(61)
    ctx, mesh = make(E, case, iop)
    q = state(mesh, rng).reshape(-1)
    tau = 0.05
    c = [np.zeros_like(q), rng.standard_normal(q.size) * 0.1]
    ref, st = krylov.phi_sum(lambda x: tau * dg.jv(mesh, q, x).reshape(-1), c, tol=1e-10, iop=iop)
    got, gst, gtr = ctx.phi(q, tau, [None, np.ascontiguousarray(c[1])])
    assert rel(got, ref) <= 1e-9
    # the same decisions: sub-steps, and Krylov dimensions within one check interval
    assert len(gtr) == len(st.trace)
    for (_, m, _, _), (_, mr, _) in zip(gtr, st.trace):
        assert abs(m - mr) <= 5


def test_phi_iom_substeps_parity(E):
    """Small m_max forces rejected attempts and sub-steps with a window of 2."""
    rng = np.random.default_rng(62)
    ctx, mesh = make(E, "burgers1d_p2", 2, m_max=10)
    q = state(mesh, rng).reshape(-1)
    tau = 0.3
    c = [rng.standard_normal(q.size) * 0.1 for _ in range(4)]
    ref, st = krylov.phi_sum(lambda x: tau * dg.jv(mesh, q, x).reshape(-1), c, tol=1e-10, m_max=10, iop=2)
    assert st.substeps > 1
    got, _, _ = ctx.phi(q, tau, [np.ascontiguousarray(x) for x in c],
                        replay=[(0, m, s, e) for (s, m, e) in st.trace])
    assert rel(got, ref) <= TOL_STEP64


def test_iom_window_covering_m_matches_full_orthogonalisation(E):
    """A window at least as long as the Krylov dimension orthogonalises against
    every previous vector: the same result as the full (DCGS2) path."""
    rng = np.random.default_rng(63)
    case = "euler2d_p4"
    ctx_f, mesh = make(E, case, 0)
    ctx_w, _ = make(E, case, 8)
    q = state(mesh, rng).reshape(-1)
    c = [None, np.ascontiguousarray(rng.standard_normal(q.size) * 0.1)]
    rep = [(0, 5, 1.0, 1.0)]
    a, _, _ = ctx_f.phi(q, 0.02, c, replay=rep)
    b, _, _ = ctx_w.phi(q, 0.02, c, replay=rep)
    assert rel(b, a) <= 1e-12


@pytest.mark.parametrize("scheme", [2, 3, 4])
@pytest.mark.parametrize("case", ["burgers1d_p2", "euler1d_p3", "euler2d_p4", "euler3d_p3"])
def test_step_iom_fp64_replayed(E, case, scheme):
    rng = np.random.default_rng(64)
    iop = 4
    ctx, mesh = make(E, case, iop, scheme=scheme)
    q = np.ascontiguousarray(state(mesh, rng))
    dt = 0.05 if mesh.eq == "euler" else 0.02
    ref, st = integrators.step(mesh, q, dt, scheme=scheme, tol=1e-10, iop=iop)
    got = q.copy()
    ctx.step(got, dt, replay=_replay_from(st))
    assert rel(got, ref) <= TOL_STEP64
    np.testing.assert_allclose(dg.totals(mesh, got), dg.totals(mesh, q), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("prec", MIXED_PRECS)
@pytest.mark.parametrize("iop", [1, 2, 4])
@pytest.mark.parametrize("scheme", [2, 3])
@pytest.mark.parametrize("case", ["burgers1d_p2", "euler2d_p4", "euler3d_p3"])
def test_step_iom_mixed_within_1e6(E, case, scheme, iop, prec):
    rng = np.random.default_rng(65)
    ctx, mesh = make(E, case, iop, prec=prec, scheme=scheme)
    q = np.ascontiguousarray(state(mesh, rng))
    dt = 0.05 if mesh.eq == "euler" else 0.02
    ref, _ = integrators.step(mesh, q, dt, scheme=scheme, tol=1e-10)
    got = q.copy()
    ctx.step(got, dt)
    assert rel(got, ref) <= TOL_MIXED


def test_iom_vortex_full_size(E):
    """64 x 64 elements, p = 4 (409,600 unknowns), window 4: one EPI2 step, FP64
    form with the oracle's decisions, and the adaptive mixed form at tol 1e-8
    against the oracle's full-Arnoldi step at 1e-10."""
    CASES["euler2d_full"] = dict(eq=2, dim=2, p=4, ne=(64, 64), lo=(0.0, 0.0), hi=(10.0, 10.0))
    ctx, mesh = make(E, "euler2d_full", 4)
    q = np.ascontiguousarray(inputs.isentropic_vortex(dg.node_coords(mesh), 0.0))
    ref, st = integrators.step(mesh, q, 0.05, tol=1e-10, iop=4)
    got = q.copy()
    ctx.step(got, 0.05, replay=_replay_from(st))
    assert rel(got, ref) <= TOL_STEP64
    full, _ = integrators.step(mesh, q, 0.05, tol=1e-10)
    for prec in MIXED_PRECS:
        ctx2, _ = make(E, "euler2d_full", 4, prec=prec, tol=1e-8)
        got2 = q.copy()
        st2, tr2 = ctx2.step(got2, 0.05)
        ctx2.close()
        assert rel(got2, full) <= TOL_MIXED, prec
        # one sub-step of about the oracle's dimension (25 at tol 1e-10 with full
        # orthogonalisation)
        assert len(tr2) == 1 and tr2[0][1] <= 40, (prec, tr2)


def test_invalid_window_rejected(E):
    for bad in (-1, E.EXPDG_MAX_IOP + 1):
        with pytest.raises(E.ExpdgError) as ei:
            E.Context(iop=bad)
        assert ei.value.status == E.EXPDG_EINVAL


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("iop", [0, 4])
def test_zero_start_vector_adaptive(E, prec, iop):
    """An adaptive phi-sum whose start vector is zero (P = 0 and c_0 = 0, or
    P = 1 with c_1 = 0 and c_0 = 0): beta and eta are formed on the device, the
    Arnoldi steps break down at once, and the result is exactly zero; a
    following non-zero solve on the same context is unaffected."""
    rng = np.random.default_rng(67)
    ctx, mesh = make(E, "euler2d_p4", iop, prec=prec)
    q = state(mesh, rng).reshape(-1)
    z = np.zeros_like(q)
    got, st, tr = ctx.phi(q, 0.05, [np.ascontiguousarray(z)])
    assert np.all(got == 0.0)
    got, st, tr = ctx.phi(q, 0.05, [None, np.ascontiguousarray(z)])
    assert np.all(got == 0.0)
    c = [np.zeros_like(q), rng.standard_normal(q.size) * 0.1]
    ref, _ = krylov.phi_sum(lambda x: 0.05 * dg.jv(mesh, q, x).reshape(-1), c, tol=1e-10, iop=iop or None)
    got, _, _ = ctx.phi(q, 0.05, [None, np.ascontiguousarray(c[1])])
    assert rel(got, ref) <= (1e-9 if prec == 0 else TOL_MIXED)


@pytest.mark.parametrize("prec", MIXED_PRECS)
def test_mixed_paired_checks_trajectory(E, prec):
    """Six EPI2 steps of the vortex on 40 x 40 elements, p = 4 (160,000
    unknowns: the FP32-operator forms' checks evaluate exp(H_{m-1}) beside
    exp(H_m) and accept on the change since m - 1), with the schedule that
    starts at the previous step's m, probes below it and retries above it.
    Float-float form: every step stays within 1e-7 of the oracle's FP64
    full-Arnoldi trajectory at tol 1e-10 (ten times the Krylov tolerance 1e-8),
    and every Krylov dimension is within 3 of the smallest one the oracle
    accepts at tol 1e-8 (the same window, a check at every m).  Mixed form
    (FP32 residual, whose rounding is the larger error there): every step within
    the 1e-6 bar."""
    CASES["euler2d_40"] = dict(eq=2, dim=2, p=4, ne=(40, 40), lo=(0.0, 0.0), hi=(10.0, 10.0))
    ctx, mesh = make(E, "euler2d_40", 4, prec=prec, tol=1e-8)
    q = np.ascontiguousarray(inputs.isentropic_vortex(dg.node_coords(mesh), 0.0))
    ref = q.copy()
    got = q.copy()
    for k in range(6):
        _, smin = integrators.step(mesh, ref, 0.08, tol=1e-8, m_step=1, iop=4)
        ref, _ = integrators.step(mesh, ref, 0.08, tol=1e-10)
        gst, gtr = ctx.step(got, 0.08)
        assert rel(got, ref) <= (1e-7 if prec == 2 else TOL_MIXED), (k, rel(got, ref))
        assert len(gtr) == 1 and len(smin.traces) == 1 and len(smin.traces[0]) == 1
        m, mr = gtr[0][1], smin.traces[0][0][1]
        if prec == 2:
            assert abs(m - mr) <= 3, (k, m, mr)


@pytest.mark.parametrize("prec", MIXED_PRECS)
@pytest.mark.parametrize("dt", [0.2, 0.3])
def test_mixed_large_krylov_dimension(E, dt, prec):
    """Long steps on the 40 x 40, p = 4 vortex (160,000 unknowns): the Krylov
    dimension passes 49, where the paired checks run on two groups of CTAs
    (or, where 16-CTA clusters do not fit, give way to the change since the
    previous check); dt = 0.2: one sub-step near m_max = 64; dt = 0.3: the
    sub-step is halved.  One mixed-form step against the oracle's FP64 step."""
    CASES["euler2d_40"] = dict(eq=2, dim=2, p=4, ne=(40, 40), lo=(0.0, 0.0), hi=(10.0, 10.0))
    ctx, mesh = make(E, "euler2d_40", 4, prec=prec, tol=1e-8)
    q = np.ascontiguousarray(inputs.isentropic_vortex(dg.node_coords(mesh), 0.0))
    ref, _ = integrators.step(mesh, q, dt, tol=1e-10)
    got = q.copy()
    gst, gtr = ctx.step(got, dt)
    assert rel(got, ref) <= TOL_MIXED
    if dt == 0.2:
        assert max(m for (_, m, _, _) in gtr) > 49
    else:
        assert gst["rejected"] >= 1 and len(gtr) >= 2
