"""The allocation-free entry point gives the same answer as the regular one.

vfpi_solve_noalloc serves callers that cannot call cudaMalloc (their device
memory belongs to another allocator, or they must never block on an
allocation): it solves a small problem from the caller's device buffers with
scratch that lives in a fixed device array inside the library.  This test calls
it through the C ABI twice in a row -- the array keeps the first call's
contents, so the second call shows that what must start empty is cleared --
and checks both results against vfpi_solve on the same problem, within the
FP32 tolerance of the other parity tests.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2201_09212_gb300 import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2201_09212_gb300 import build, vfpi  # noqa: E402

TOL = 1e-5   # the FP32 tolerance of tests/test_gpu_parity.py


def close(a, b, rtol=TOL):
    a, b = np.asarray(a, float), np.asarray(b, float)
    scale = max(np.abs(b).max(), 1e-300)
    return np.abs(a - b).max() / scale <= rtol


def noalloc_solve(sc, v0, theta_th, l_max, norm=0):
    L = vfpi.lib()
    dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()
    rp, ci, va = dev(sc.row_ptr, np.int32), dev(sc.col_idx, np.int32), dev(sc.vals, np.float32)
    b = dev(sc.b, np.float32)
    ni, nj = dev(sc.node_i, np.int32), dev(sc.node_j, np.int32)
    R, mu, phi = dev(sc.R, np.float32), dev(sc.mu, np.float32), dev(sc.phi, np.float32)
    v_in = dev(v0, np.float32)
    v_out = torch.full_like(v_in, float("nan"))
    lam = torch.full((3 * sc.n_c,), float("nan"), dtype=torch.float32, device="cuda")
    bsr = vfpi._Bsr(sc.n_nodes, sc.nnzb, rp.data_ptr(), ci.data_ptr(), va.data_ptr())
    con = vfpi._Contacts(sc.n_c, ni.data_ptr(), nj.data_ptr(), R.data_ptr(), mu.data_ptr(),
                         phi.data_ptr())
    iters = C.c_int32(-1)
    theta = C.c_double(-1.0)
    torch.cuda.synchronize()
    st = L.vfpi_solve_noalloc(C.byref(bsr), b.data_ptr(), C.byref(con), C.c_double(theta_th),
                              l_max, norm, v_in.data_ptr(), v_out.data_ptr(), lam.data_ptr(),
                              C.byref(iters), C.byref(theta), None)
    assert st in (vfpi.VFPI_OK, vfpi.VFPI_NOT_CONVERGED), (st, L.vfpi_noalloc_last_error())
    return v_out.cpu().numpy(), lam.cpu().numpy(), iters.value, theta.value, st


def regular_solve(sc, v0, theta_th, l_max, norm="abs"):
    with vfpi.Solver.from_scene(sc, dtype="f32", theta_th=theta_th, l_max=l_max, norm=norm) as s:
        r = s.solve(np.asarray(v0, np.float32))
    return r


@pytest.mark.parametrize("case", ["lattice", "random_with_d_contacts"])
def test_noalloc_matches_vfpi_solve_on_two_calls_in_a_row(case):
    build.build()
    if case == "lattice":
        sc = scenes.small_lattice(np.float32)
        first = dict(theta_th=0.0, l_max=120)
        second = dict(theta_th=1e-7, l_max=3000)
    else:
        rng = np.random.default_rng(77)
        sc = scenes.random_problem(rng, 150, 20, d_contacts=10, density=0.04, couple=0.5,
                                   dtype=np.float32)
        first = dict(theta_th=0.0, l_max=40)
        second = dict(theta_th=1e-6, l_max=2000)
    starts = [sc.v0, 0.5 * sc.v0 + 0.01]
    for v0, kw in zip(starts, (first, second)):
        v, lam, iters, theta, st = noalloc_solve(sc, v0, **kw)
        ref = regular_solve(sc, v0, **kw)
        assert iters == ref.iters, (iters, ref.iters)
        assert st == ref.status
        assert close(v, ref.v) and np.isfinite(v).all()
        assert close(lam.reshape(-1, 3), np.asarray(ref.lam).reshape(-1, 3))
        assert abs(theta - ref.theta) <= TOL * (ref.theta + np.linalg.norm(ref.v))


def test_noalloc_rejects_problems_over_its_limit():
    L = vfpi.lib()
    x = torch.zeros(16, dtype=torch.float32, device="cuda")
    bsr = vfpi._Bsr(4097, 4097, x.data_ptr(), x.data_ptr(), x.data_ptr())
    st = L.vfpi_solve_noalloc(C.byref(bsr), x.data_ptr(), None, C.c_double(1e-6), 10, 0,
                              x.data_ptr(), x.data_ptr(), None, None, None, None)
    assert st == -1
    assert b"4096" in L.vfpi_noalloc_last_error()
    # host arrays are refused too (the call never copies or allocates)
    h = np.zeros(16, dtype=np.float32)
    bsr = vfpi._Bsr(2, 2, h.ctypes.data, h.ctypes.data, h.ctypes.data)
    st = L.vfpi_solve_noalloc(C.byref(bsr), h.ctypes.data, None, C.c_double(1e-6), 10, 0,
                              h.ctypes.data, h.ctypes.data, None, None, None, None)
    assert st == -1
