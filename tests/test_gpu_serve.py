"""The serving loop on the GPU: requests of several shapes and video
sequences overlap on the device; every result must be the same as the same
frame solved alone (bit for bit for cold starts; within the FP32 solve
tolerance for warm starts, which begin from the previous frame) and must meet
the residual target, checked by the oracle."""
import numpy as np
import pytest

from oracle import inpaint_ref as ref

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2110_03946_gb300.inpaint import Inpainter  # noqa: E402
from paper_2110_03946_gb300.serve import CudaBackend, Server, make_pool, poisson_stream  # noqa: E402

TOL_U = 0.05
PRM = dict(block=32, overlap=3, local_cg_iters=16, robin_p=0.15, levels=3, coarse_tol=3e-3)


def test_serving_results_equal_alone_and_in_the_mix():
    shapes = [(96, 128, 3), (64, 80, 1), (120, 90, 3)]
    pool = make_pool(shapes, n_frames=4, n_masks=3, density_range=(0.03, 0.08), seed=5)
    reqs = poisson_stream(400.0, 0.06, shapes, [0.5, 0.25, 0.25], 4, 10, pool)
    assert len(reqs) >= 12
    backend = CudaBackend(PRM, tol=1e-6)
    srv = Server(backend, hbm_budget=1 << 30)
    got = {}

    def on_result(r):
        got[r.rid] = (r.output.clone(), r.warm, r.status)

    res, m = srv.run(reqs, realtime=False, on_result=on_result)
    srv.close()
    assert m["failures"] == 0 and len(got) == len(reqs)
    assert m["warm_starts"] > 0 and m["slots_created"] >= len(shapes)
    for rq in reqs:
        u, warm, status = got[rq.rid]
        u = u.numpy()
        f = rq.values.numpy().astype(np.float64)
        mask = rq.mask.numpy()
        with Inpainter(mask, f, precision="fp32", **PRM) as ip:
            alone = ip.solve(1e-6).cpu().numpy()
        if warm:
            assert np.max(np.abs(u - alone)) <= TOL_U
        else:
            assert np.array_equal(u, alone)
        assert np.all(ref.rel_residual(u.astype(np.float64), f, mask) <= 1e-6)
        assert np.max(np.abs(u - ref.solve_direct(f, mask))) <= TOL_U
