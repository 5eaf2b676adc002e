"""The allocation-free entry point gives the same answer as the regular one.

vfpi_solve_noalloc serves callers that cannot call cudaMalloc (their device
memory belongs to another allocator, or they must never block on an
allocation): it solves a small problem from the caller's device buffers with
scratch that lives in a fixed device array inside the library.  This test calls
it through the C ABI twice in a row -- the array keeps the first call's
contents, so the second call shows that what must start empty is cleared --
and checks both results against vfpi_solve on the same problem, within the
FP32 tolerance of the other parity tests, and against the FP64 oracle.  The
inputs it must refuse (a bad row_ptr, an out-of-range node or column index, a
node in two contacts) are checked on the device before any block is read, so
those cases run no access out of range; each returns its status and leaves
the outputs unwritten.
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


def noalloc_call(sc, v0, theta_th, l_max, norm=0, row_ptr=None, col_idx=None, node_i=None,
                 node_j=None):
    """One call through the C ABI; returns (status, v_out, lambda_out, iters, theta).
    The optional arrays replace the scene's (to plant invalid inputs)."""
    L = vfpi.lib()
    dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()
    pick = lambda a, d: d if a is None else a
    rp = dev(pick(row_ptr, sc.row_ptr), np.int32)
    ci = dev(pick(col_idx, sc.col_idx), np.int32)
    va = dev(sc.vals, np.float32)
    b = dev(sc.b, np.float32)
    ni, nj = dev(pick(node_i, sc.node_i), np.int32), dev(pick(node_j, sc.node_j), np.int32)
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
    return st, v_out.cpu().numpy(), lam.cpu().numpy(), iters.value, theta.value


def noalloc_solve(sc, v0, theta_th, l_max, norm=0):
    st, v, lam, iters, theta = noalloc_call(sc, v0, theta_th, l_max, norm)
    assert st in (vfpi.VFPI_OK, vfpi.VFPI_NOT_CONVERGED), (st, vfpi.lib().vfpi_noalloc_last_error())
    return v, lam, iters, theta, st


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


def _oracle_case(case):
    if case == "lattice":
        return scenes.small_lattice(np.float32)
    rng = np.random.default_rng(77)
    return scenes.random_problem(rng, 150, 20, d_contacts=10, density=0.04, couple=0.5,
                                 dtype=np.float32)


@pytest.mark.parametrize("case", ["lattice", "random_with_d_contacts"])
def test_noalloc_matches_the_fp64_oracle(case):
    """Against the FP64 oracle (Alg. 1 + Alg. 2 on the same FP32 inputs): after a
    fixed number of sweeps element by element, and at convergence within
    north-star's bar (relative velocity error <= 1e-5, scaled Signorini-Coulomb
    residual <= 1e-6)."""
    from oracle import vfpi as ov
    from oracle.checks import scc_residual
    from tests.conftest import oracle_problem
    build.build()
    sc = _oracle_case(case)
    P = oracle_problem(sc)
    w = ov.frobenius_w(P)
    v0 = np.asarray(sc.v0, np.float32).astype(np.float64)
    for k in (1, 10):
        v, lam, iters, _, st = noalloc_solve(sc, sc.v0, 0.0, k)
        ref = ov.solve(P, w, v0, theta_th=0.0, l_max=k)
        assert iters == k and st == vfpi.VFPI_NOT_CONVERGED
        assert close(v, ref.v), k
        assert close(lam.reshape(-1, 3), ref.lam), k
    # the same stop test on both sides (absolute theta, as the lattice's and
    # the random problem's second calls above use it)
    th = 1e-7 if case == "lattice" else 1e-6
    v, lam, iters, theta, st = noalloc_solve(sc, sc.v0, th, 5000)
    assert st == vfpi.VFPI_OK and theta < th
    ref = ov.solve(P, w, v0, theta_th=th, l_max=200000)
    assert ref.converged and abs(iters - ref.iters) <= 1, (iters, ref.iters)
    if iters != ref.iters:      # theta within rounding of the threshold on one side
        ref = ov.solve(P, w, v0, theta_th=0.0, l_max=iters)
    err = np.linalg.norm(v.astype(float) - ref.v) / np.linalg.norm(ref.v)
    assert err <= 1e-5, err
    assert np.abs(v - ref.v).max() <= 1e-5 * np.abs(ref.v).max()
    assert scc_residual(P, v.astype(float), lam.astype(float).reshape(-1, 3)) <= 1e-6


def test_noalloc_rejects_invalid_inputs_before_reading_a_block():
    """Each invalid input is found by the kernel's checks before any loop over
    a row's blocks (so nothing is read out of range): bad row pointers, a node
    or column index past the last node, a node claimed by two contacts, a
    D-contact joining a node to itself.  The call returns the status, the
    outputs stay as they were, and the next valid call is unaffected."""
    build.build()
    L = vfpi.lib()
    sc = _oracle_case("random_with_d_contacts")
    N, nnzb = sc.n_nodes, sc.nnzb
    assert (sc.node_j >= 0).any() and (sc.node_j < 0).any()
    s_idx = int(np.nonzero(sc.node_j < 0)[0][0])
    d_idx = int(np.nonzero(sc.node_j >= 0)[0][0])
    rp_end = sc.row_ptr.copy()
    rp_end[-1] = nnzb - 1                                 # does not end at nnzb
    rp_start = sc.row_ptr.copy()
    rp_start[0] = 1                                       # does not start at 0
    rp_back = sc.row_ptr.copy()
    rp_back[2] = rp_back[1] - 1                           # row 1 has a negative length
    ci = sc.col_idx.copy()
    ci[nnzb // 2] = N                                     # column past the last node
    ni_out = sc.node_i.copy()
    ni_out[s_idx] = N                                     # node past the last node
    ni_twice = sc.node_i.copy()
    other = [m for m in range(sc.n_c) if m != s_idx][0]
    ni_twice[other] = sc.node_i[s_idx]                    # one node, two contacts
    nj_self = sc.node_j.copy()
    nj_self[d_idx] = sc.node_i[d_idx]                     # D-contact from a node to itself
    cases = [
        ("row_ptr end", dict(row_ptr=rp_end), vfpi.STATUS_CODES["VFPI_ERR_INVALID_ARG"], b"row_ptr"),
        ("row_ptr start", dict(row_ptr=rp_start), vfpi.STATUS_CODES["VFPI_ERR_INVALID_ARG"], b"row_ptr"),
        ("row_ptr order", dict(row_ptr=rp_back), vfpi.STATUS_CODES["VFPI_ERR_INVALID_ARG"], b"row_ptr"),
        ("column index", dict(col_idx=ci), vfpi.STATUS_CODES["VFPI_ERR_INVALID_ARG"], b"index"),
        ("node index", dict(node_i=ni_out), vfpi.STATUS_CODES["VFPI_ERR_INVALID_ARG"], b"index"),
        ("node in two contacts", dict(node_i=ni_twice),
         vfpi.STATUS_CODES["VFPI_ERR_CONTACT_OVERLAP"], b"two contacts"),
        ("D-contact to itself", dict(node_j=nj_self),
         vfpi.STATUS_CODES["VFPI_ERR_CONTACT_OVERLAP"], b"two contacts"),
    ]
    for name, kw, want, msg in cases:
        st, v, lam, iters, _ = noalloc_call(sc, sc.v0, 1e-6, 50, **kw)
        assert st == want, (name, st)
        assert msg in L.vfpi_noalloc_last_error(), (name, L.vfpi_noalloc_last_error())
        assert np.isnan(v).all() and np.isnan(lam).all(), name
        assert iters == 0, name
    # the shared array carries nothing over from the refused calls
    ref = regular_solve(sc, sc.v0, theta_th=1e-6, l_max=2000)
    v, lam, iters, _, st = noalloc_solve(sc, sc.v0, 1e-6, 2000)
    assert iters == ref.iters and st == ref.status
    assert close(v, ref.v) and close(lam.reshape(-1, 3), np.asarray(ref.lam).reshape(-1, 3))
