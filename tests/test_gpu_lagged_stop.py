"""The TMA ring kernel's lagged stop test (Alg. 1): each sweep's CTA partials
are added while the next sweep's grid barrier completes, so the stop test of
sweep l runs one sweep behind and the sweep after a stop is discarded.  The
outcome must be the plain kernel's: v_hat, lambda, lambda* bit for bit, the
same iteration count and status, and theta up to the order in which another
launch shape adds its CTA partials -- for a converged solve, for l_max reached (odd and
even), for a stop at the first sweep, for l_max = 1 (no lag), and for two
solves in a row on the same context (the odd sweeps' lambda buffers)."""
import numpy as np
import pytest

from paper_2201_09212_gb300 import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2201_09212_gb300 import vfpi  # noqa: E402

CASES = [dict(theta_th=1e-6, l_max=300), dict(theta_th=-1.0, l_max=7),
         dict(theta_th=-1.0, l_max=8), dict(theta_th=-1.0, l_max=2), dict(theta_th=1e9, l_max=50),
         dict(theta_th=-1.0, l_max=1)]


def run(sc, variant, starts, **kw):
    out = []
    with vfpi.Solver.from_scene(sc, norm="rms", force_path=1, **kw) as s:
        s.configure_launch(variant, 0, 0)
        for v in starts:
            r = s.solve(v)
            out.append((r.v, s.get_lambda(), s.get_lambda_star(), r.iters, r.theta, r.status))
    return out


@pytest.mark.parametrize("scene", ["fem", "terrain"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_lagged_stop_equals_the_plain_kernel(scene, case):
    sc = (scenes.fem_block_scene(16, 16, 6, seed=3, dtype=np.float32) if scene == "fem"
          else scenes.terrain_lattice(dims=(40, 36, 6)))
    starts = [sc.v0, (np.asarray(sc.v0) * 0.5).astype(sc.v0.dtype)]
    ref = run(sc, 7, starts, **CASES[case])
    for var in (26, 27, 8):
        got = run(sc, var, starts, **CASES[case])
        for g, r in zip(got, ref):
            for a, b in zip(g[:3], r[:3]):
                assert np.array_equal(a, b), (var, CASES[case])
            assert g[3] == r[3] and g[5] == r[5], (var, CASES[case], g[3:], r[3:])
            # theta: the same sweep's, summed over another grid of CTA partials
            assert g[4] == pytest.approx(r[4], rel=1e-9, abs=0.0), (var, CASES[case])
