"""coil_apply_operator_static: the operator product for callers that cannot
allocate device memory once they are running (stream capture, real-time
loops with fixed memory, capped processes).  It must give what
coil_apply_operator gives, call after call, with the shared scratch array
reused in between.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2403_07666_b300 import build as B
from paper_2403_07666_b300 import workloads as wl
from tests.gpu_common import rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
def test_static_apply_matches_regular_apply_twice(precision, tol):
    import torch
    from paper_2403_07666_b300.coil import Coil
    w = wl.random_coil(71, 5, 7, 4)                      # 560 elements, ragged row tiles
    rng = np.random.default_rng(9)
    p1 = rng.standard_normal(w.n_elem)
    p2 = rng.standard_normal(w.n_elem) * 3.0
    with Coil.from_workload(w, precision=precision) as c:
        ref1 = c.apply_operator(p1)
        ref2 = c.apply_operator(p2)
        dev = torch.device("cuda", 0)
        d_p1 = torch.tensor(p1, dtype=torch.float64, device=dev)
        d_p2 = torch.tensor(p2, dtype=torch.float64, device=dev)
        d_y1 = torch.full((w.n_elem,), float("nan"), dtype=torch.float64, device=dev)
        d_y2 = torch.full((w.n_elem,), float("nan"), dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream(dev)
        c.apply_operator_static(d_p1.data_ptr(), d_y1.data_ptr(), stream.cuda_stream)
        c.apply_operator_static(d_p2.data_ptr(), d_y2.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize(dev)
        y1 = d_y1.cpu().numpy()
        y2 = d_y2.cpu().numpy()
    assert rel(y1, ref1) < tol
    assert rel(y2, ref2) < tol
