"""poisson_solve_noalloc: the Poisson entry point for callers that cannot
allocate device memory (no workspace; the library's fixed device scratch is
used instead).  Called through the C ABI and compared with poisson_solve,
which runs the same solver in a caller workspace, on two calls in a row (the
second call must not be affected by what the first left in the shared
scratch).  Collected last so that a failure here cannot hide other tests."""
import ctypes as C

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_14494_gb300 import build
    build.build()


def _noalloc(P, pc, rho, phi, mask, E, rtol):
    st = P.poisson_stats()
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = P.lib().poisson_solve_noalloc(C.byref(pc), C.c_void_p(rho.data_ptr()), C.c_void_p(mask.data_ptr()),
                                       C.c_void_p(phi.data_ptr()), *(C.c_void_p(e.data_ptr()) for e in E), rtol, 100,
                                       C.byref(st), s)
    torch.cuda.synchronize()
    return rc, st


@pytest.mark.parametrize("precision", [64, 32])
def test_noalloc_matches_workspace_solve_twice(precision):
    """Both precisions: 64 keeps the float64 CG vectors in the scratch, 32 the
    float-pair potential, the float32 CG vectors and the loop counters."""
    from paper_2110_14494_gb300 import picmcc as P
    grid = W.grid_spec(48, 40, 64, 4e-5)
    V0 = 1500.0
    rtol = 1e-9 if precision == 64 else 1e-8
    mask = torch.as_tensor(W.needle_mask(grid, 0.9e-3, 0.15e-3)).cuda()
    pc = P.poisson_config(48, 40, 64, 4e-5, 0.0, V0, V0, precision)
    for call, off in enumerate((3, 4)):
        rho = torch.as_tensor(W.random_rho(grid, off, 5e-2)).cuda()
        ref_phi = torch.zeros_like(rho)
        refE = tuple(torch.zeros(rho.shape, dtype=torch.float32, device="cuda") for _ in range(3))
        cyc, rel = P.poisson_solve(grid, rho, ref_phi, mask=mask, E=refE, v_lo=0.0, v_hi=V0, v_mask=V0, rtol=rtol,
                                   max_cycles=100, precision=precision)
        phi = torch.zeros_like(rho)
        E = tuple(torch.zeros(rho.shape, dtype=torch.float32, device="cuda") for _ in range(3))
        rc, st = _noalloc(P, pc, rho, phi, mask, E, rtol)
        assert rc == P.PIC_OK, call
        assert st.rel_res <= rtol and abs(st.cycles - cyc) <= 1, (call, st.cycles, cyc)
        a, b = phi.cpu().numpy(), ref_phi.cpu().numpy()
        assert np.abs(a - b).max() <= rtol * np.abs(b).max(), call
        for x, y in zip(E, refE):
            assert torch.equal(x, y) or float((x - y).abs().max()) <= 1e-6 * float(y.abs().max()), call


def test_noalloc_rejects_grids_beyond_its_scratch():
    from paper_2110_14494_gb300 import picmcc as P
    pc = P.poisson_config(256, 256, 256, 1e-5, 0.0, 1.0, 1.0)
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = P.lib().poisson_solve_noalloc(C.byref(pc), C.c_void_p(dummy.data_ptr()), None, C.c_void_p(dummy.data_ptr()),
                                       None, None, None, 1e-6, 10, None, None)
    assert rc == P.PIC_ERR_CAPACITY
