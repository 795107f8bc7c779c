"""Parity on the stand-ins for the paper's timing meshes (Section 3.2): the
smallest and the largest of the six node counts, only the bottom of the
surface held at 37 degC and the rest insulated, 2000 steps of 0.005 s (the
paper's run), against the FP64 oracle for all 2000 steps: FP64 within
1e-9 degC, FP32+Kahan within 1e-3 degC, on the persistent and the staged
tiled kernels; temperature-dependent laws at both sizes, constant ones at
the smallest."""
import pytest

from oracle import Oracle
from synth.scenarios import paper_size_ellipsoid

from gpu_util import ff, max_abs, run_gpu

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-9, 1e-3
DT, STEPS = 0.005, 2000


@pytest.mark.parametrize("nodes,td", [(1445, True), (1445, False), (7872, True)])
def test_paper_size_mesh_full_run_against_the_oracle(nodes, td):
    f = ff()
    p = paper_size_ellipsoid(nodes, temperature_dependent=td).problem
    ref = Oracle(p).run(DT, STEPS)
    assert ref.max() > 60.0                      # the insulated mesh heats well past the reference 37 degC
    for kern in (f.KERNEL_PERSISTENT, f.KERNEL_TILED_STAGED):
        for prec, tol in ((f.FP64, TOL64), (f.FP32_KAHAN, TOL32)):
            T, info = run_gpu(p, DT, STEPS, prec, kernel=kern)
            err = max_abs(T, ref)
            print(f"{p.n_nodes} nodes {'TD' if td else 'TI'} kernel {kern} prec {prec}: max|dT| = {err:.3e} "
                  f"(T up to {ref.max():.2f})")
            assert err <= tol
