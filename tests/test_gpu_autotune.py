"""GPU checks of the autotuner (pp_autotune): after it picks the degree and
the stencil kernel's block shape, operator applications and solves still
match the FP64 oracle at the parity tolerances (operator 2e-13 double-word /
4e-7 FP32; solves 1e-10)."""
import numpy as np
import pytest

import synth
from oracle import exact, operators as ops
from tests.libpp import load

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


@pytest.mark.parametrize("prec,op_tol", [(1, 2e-13), (2, 4e-7)], ids=["dw", "mixed"])
@pytest.mark.parametrize("kind,dims", [("laplace3d", (48, 40, 36)), ("laplace2d", (300, 256)),
                                       ("convdiff", (40, 36, 30))])
def test_autotuned_handle_parity(kind, dims, prec, op_tol):
    pp = load()
    sk = {"laplace3d": pp.PP_LAPLACE3D7, "laplace2d": pp.PP_LAPLACE2D5, "convdiff": pp.PP_CONVDIFF3D7_UPWIND}[kind]
    h = pp.pp_create_stencil(sk, dims, [0.5] if kind == "convdiff" else None)
    try:
        o = pp.pp_default_opts()
        o.precision = prec
        pp.pp_set_opts(h, o)
        d = pp.pp_autotune(h, 1e-10, 64)
        assert 0 <= d <= 64
        n = int(np.prod(dims))
        A = ops.convdiff(dims, 0.5) if kind == "convdiff" else ops.laplace(dims)
        x = synth.rhs(n, 3)
        y = torch.empty(n, dtype=torch.float64, device="cuda")
        pp.pp_op_apply(h, torch.from_numpy(x).cuda(), y)
        torch.cuda.synchronize()
        assert rel(y.cpu().numpy(), A @ x) < op_tol
        if kind != "convdiff":
            b = synth.rhs(n, 0)
            st = pp.pp_apply(h, -1, torch.from_numpy(b).cuda(), y, m_max=600, tol=1e-11)
            torch.cuda.synchronize()
            assert st.status == pp.PP_OK
            assert rel(y.cpu().numpy(), exact.separable_fun(dims, b, -0.5)) < 1e-10
    finally:
        pp.pp_destroy(h)
