"""CTA size (tile class) of the FP32 operator apply (mixed and float-float
forms): the three classes give bit-identical results (a node's arithmetic
does not depend on which nodes share its CTA), steps with a forced class meet
those forms' bar against the oracle, and the autotuned choice is one of the
three and is reused for a second context of the same mesh."""
import numpy as np
import pytest

from oracle import dg, integrators
from tests.test_gpu_parity import CASES, MIXED_PRECS, TOL_MIXED, rel, state

pytestmark = pytest.mark.gpu

TILES = (1, 2, 3)  # EXPDG_TILE_256, _128, _512


@pytest.fixture(scope="module")
def E():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_01316_gb300 import expdg
    return expdg


def make(E, case, tile, flux=0, prec=1, **kw):
    c = CASES[case]
    ctx = E.Context(eq=c["eq"], dim=c["dim"], p=c["p"], ne=list(c["ne"]) + [1] * (3 - c["dim"]),
                    lo=list(c["lo"]) + [0.0] * (3 - c["dim"]), hi=list(c["hi"]) + [1.0] * (3 - c["dim"]),
                    prec=prec, scheme=2, krylov_tol=1e-10, m_max=64, m_step=5, max_substeps=32, gamma=1.4,
                    iop=4, tile=tile, flux=flux, **kw)
    mesh = dg.Mesh(dim=c["dim"], p=c["p"], ne=c["ne"], lo=c["lo"], hi=c["hi"],
                   eq="burgers" if c["eq"] == 1 else "euler", flux="roe" if flux else "lf")
    return ctx, mesh


@pytest.mark.parametrize("prec", MIXED_PRECS)
@pytest.mark.parametrize("flux", [0, 1])
@pytest.mark.parametrize("case", ["euler1d_p3", "euler2d_p4", "euler2d_p1", "euler2d_p7", "euler3d_p3", "euler3d_p2",
                                  "burgers1d_p2"])
def test_tiles_bit_identical(E, case, flux, prec):
    if flux and CASES[case]["eq"] == 1:
        pytest.skip("Roe flux: Euler only")
    rng = np.random.default_rng(101)
    outs = []
    for t in TILES:
        ctx, mesh = make(E, case, t, flux, prec=prec)
        assert ctx.tile == t
        if not outs:
            q = np.ascontiguousarray(state(mesh, rng))
            v = np.ascontiguousarray(rng.standard_normal(q.shape))
        outs.append(ctx.jv(q, v))
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])


@pytest.mark.parametrize("prec", MIXED_PRECS)
@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("case", ["euler2d_p4", "euler3d_p3"])
def test_tile_step_mixed(E, case, tile, prec):
    rng = np.random.default_rng(102)
    ctx, mesh = make(E, case, tile, prec=prec)
    q = np.ascontiguousarray(state(mesh, rng))
    ref, _ = integrators.step(mesh, q, 0.05, tol=1e-10)
    got = q.copy()
    ctx.step(got, 0.05)
    assert rel(got, ref) <= TOL_MIXED


@pytest.mark.parametrize("prec", MIXED_PRECS)
def test_autotuned_tile_is_valid_and_cached(E, prec):
    a, _ = make(E, "euler2d_p4", 0, prec=prec)
    b, _ = make(E, "euler2d_p4", 0, prec=prec)
    assert a.tile in TILES and b.tile == a.tile
    f64 = E.Context(dim=2, p=4, ne=[6, 5, 1], prec=0)
    assert f64.tile == 1  # the FP64 form keeps the default size


def test_invalid_tile_rejected(E):
    for bad in (-1, 6):
        with pytest.raises(E.ExpdgError) as ei:
            E.Context(tile=bad)
        assert ei.value.status == E.EXPDG_EINVAL
