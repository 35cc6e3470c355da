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


def _static_apply(c, ps):
    """The static entry point on each vector of ``ps`` in a row, outputs
    pre-filled with NaN so that an element it never writes shows."""
    import torch
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    outs = []
    for p in ps:
        d_p = torch.tensor(p, dtype=torch.float64, device=dev)
        d_y = torch.full((p.size,), float("nan"), dtype=torch.float64, device=dev)
        c.apply_operator_static(d_p.data_ptr(), d_y.data_ptr(), stream.cuda_stream)
        outs.append((d_p, d_y))
    torch.cuda.synchronize(dev)
    return [y.cpu().numpy() for _, y in outs]


# FP64: the same products in another order; FP32 / BF16 storage: the same FP32
# products of the same stored entries, summed in another order
TOL = {"fp64": 1e-12, "fp32": 2e-6, "bf16": 5e-6}


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
def test_static_apply_matches_regular_apply_twice(precision):
    from paper_2403_07666_b300.coil import Coil
    w = wl.random_coil(71, 5, 7, 4)                      # 560 elements, ragged row tiles
    rng = np.random.default_rng(9)
    p1 = rng.standard_normal(w.n_elem)
    p2 = rng.standard_normal(w.n_elem) * 3.0
    with Coil.from_workload(w, precision=precision) as c:
        ref1 = c.apply_operator(p1)
        ref2 = c.apply_operator(p2)
        y1, y2 = _static_apply(c, [p1, p2])
    assert rel(y1, ref1) < TOL[precision]
    assert rel(y2, ref2) < TOL[precision]


def test_static_apply_larger_coil_then_smaller_coil():
    """The scratch keeps the larger coil's input past the smaller coil's N;
    the smaller coil's product must not see it."""
    from paper_2403_07666_b300.coil import Coil
    big = wl.random_coil(72, 6, 9, 4)                    # 864 elements
    small = wl.random_coil(73, 3, 5, 4)                  # 240 elements
    rng = np.random.default_rng(10)
    pb = 1.0 + rng.random(big.n_elem) * 1e3
    ps = rng.standard_normal(small.n_elem)
    with Coil.from_workload(big, precision="fp32") as cb, Coil.from_workload(small, precision="fp32") as cs:
        yb = _static_apply(cb, [pb])[0]
        ys1, ys2 = _static_apply(cs, [ps, ps])
        refb = cb.apply_operator(pb)
        refs = cs.apply_operator(ps)
    assert rel(yb, refb) < TOL["fp32"]
    assert rel(ys1, refs) < TOL["fp32"]
    assert np.array_equal(ys1, ys2)


def test_static_apply_long_rows():
    """A 19,968-element coil: rows of about 20k FP32 terms, where a single
    FP32 partial per lane would drift from the regular apply."""
    from paper_2403_07666_b300.coil import Coil
    w = wl.profile_coil()
    rng = np.random.default_rng(11)
    p1 = 0.5 + rng.random(w.n_elem)
    p2 = rng.standard_normal(w.n_elem)
    with Coil.from_workload(w, precision="fp32") as c:
        ref1 = c.apply_operator(p1)
        ref2 = c.apply_operator(p2)
        y1, y2 = _static_apply(c, [p1, p2])
    assert rel(y1, ref1) < 2e-6
    assert rel(y2, ref2) < 2e-5
