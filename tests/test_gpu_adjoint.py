"""GPU adjoint (coil_adjoint) against central finite differences of the FP64
oracle: gradients of a magnetization-loop loss with respect to the creep
exponent n, the strain coefficient C_eps and the per-element Jc factor, also
with the Lorentz hoop strain coupling J and B_z into Jc."""
import numpy as np
import pytest

import oracle
from paper_2403_07666_b300 import build as B
from paper_2403_07666_b300 import workloads as wl

pytestmark = pytest.mark.gpu

K = 40


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


def _loop_coil(thermal=1, transport=0, Y_eff=0.0):
    """Free loops (or a transport ramp) under a triangular applied field, past
    penetration, with heating: the field-loop calibration case."""
    mtl = dict(wl.MATERIAL, Jc0=2e8, thermal=thermal, Y_eff=Y_eff)
    w = wl.random_coil(81, 3, 4, 4, ramp_rate=2e4 if transport else 0.0, I_max=1e9, dt=1e-4,
                       Ba_rate=4.0, Ba_max=0.02, Ba_waveform=2, material=mtl)
    w.geometry["transport"] = transport
    return w


def _oracle_moments(w, f=None, n=None, ce=None):
    o = oracle.build(w.geometry, w.material, w.jc_factor if f is None else f, w.strain, w.mat)
    if n is not None:
        o.p["n"] = n
    if ce is not None:
        o.p["C_eps"] = ce
    return np.array([o.step(w.drive)[3] for _ in range(K)])


@pytest.mark.parametrize("thermal,transport,Y_eff", [(1, 0, 0.0), (0, 1, 0.0), (1, 0, 5e7), (0, 1, 5e7)])
def test_adjoint_matches_oracle_finite_differences(thermal, transport, Y_eff):
    from paper_2403_07666_b300.coil import Coil
    w = _loop_coil(thermal, transport, Y_eff)
    target = _oracle_moments(w, f=w.jc_factor * 1.05, n=27.0)

    def loss(m):
        return np.sum((m - target) ** 2)

    with Coil.from_workload(w, rtol=1e-11) as c:
        s0 = c.save_state()
        c.step(K, w.drive)
        m = c.diag(0, K)[:, 3]
        c.load_state(s0)
        gf, gn, gc = c.adjoint(K, w.drive, 2.0 * (m - target), ckpt_every=10)
        # a different checkpoint spacing (uneven last segment) gives the same gradient
        c.load_state(s0)
        gf2, gn2, gc2 = c.adjoint(K, w.drive, 2.0 * (m - target), ckpt_every=7)
    assert np.array_equal(gf, gf2) and gn == gn2 and gc == gc2
    # central differences of the oracle (direct solves, FP64)
    n0, c0 = w.material["n"], w.material["C_eps"]
    hn, hc = 1e-6 * n0, 1e-6 * c0
    fd_n = (loss(_oracle_moments(w, n=n0 + hn)) - loss(_oracle_moments(w, n=n0 - hn))) / (2 * hn)
    fd_c = (loss(_oracle_moments(w, ce=c0 + hc)) - loss(_oracle_moments(w, ce=c0 - hc))) / (2 * hc)
    assert abs(gn / fd_n - 1) < 1e-4, (gn, fd_n)
    assert abs(gc / fd_c - 1) < 1e-4, (gc, fd_c)
    rng = np.random.default_rng(5)
    for _ in range(2):
        v = rng.standard_normal(w.n_elem)
        h = 1e-6
        fd = (loss(_oracle_moments(w, f=w.jc_factor * (1 + h * v)))
              - loss(_oracle_moments(w, f=w.jc_factor * (1 - h * v)))) / (2 * h)
        ad = np.sum(gf * w.jc_factor * v)
        assert abs(ad / fd - 1) < 1e-4, (ad, fd)


def test_autograd_function_backward():
    import torch
    from paper_2403_07666_b300.autograd import CoilMoments
    from paper_2403_07666_b300.coil import Coil
    w = _loop_coil(1, 0)
    target = torch.from_numpy(_oracle_moments(w, f=w.jc_factor * 1.05, n=27.0))
    with Coil.from_workload(w, rtol=1e-11) as c:
        f = torch.tensor(w.jc_factor, dtype=torch.float64, requires_grad=True)
        n = torch.tensor(30.0, dtype=torch.float64, requires_grad=True)
        ce = torch.tensor(900.0, dtype=torch.float64, requires_grad=True)
        m = CoilMoments.apply(c, w.drive, K, 10, f, n, ce)
        L = torch.sum((m - target) ** 2)
        L.backward()
        assert c.info().steps == K
        c2 = Coil.from_workload(w, rtol=1e-11)
        s0 = c2.save_state()
        c2.step(K, w.drive)
        mm = c2.diag(0, K)[:, 3]
        c2.load_state(s0)
        gf, gn, gc = c2.adjoint(K, w.drive, 2.0 * (mm - target.numpy()), ckpt_every=10)
        c2.close()
    assert np.allclose(f.grad.numpy(), gf, rtol=1e-12, atol=0)
    assert abs(n.grad.item() - gn) <= 1e-12 * abs(gn)


def _soft_max_power(P, scale):
    """Smooth quench-onset loss: the soft maximum of the Joule-power series,
    scale log sum exp(P_k / scale), and its derivative (the softmax weights)."""
    z = P / scale
    zm = np.max(z)
    wts = np.exp(z - zm)
    L = scale * (zm + np.log(np.sum(wts)))
    return L, wts / np.sum(wts)


# FP64 form: the discrete adjoint of the same step, solved to rtol 1e-11.
# Tensor-core form: FP32-class operator and FP32 pointwise chain in the forward
# states and the transposed solves (gradients within about 1e-4 of the FP64
# ones, as the mixed-precision bounds allow).
@pytest.mark.parametrize("form,tol", [("fp64", 1e-6), ("toeplitz_tc", 1e-3)])
@pytest.mark.parametrize("thermal,transport,Y_eff", [(1, 0, 0.0), (1, 1, 5e7)])
def test_adjoint_matches_tangent_linear_oracle(form, tol, thermal, transport, Y_eff):
    """coil_adjoint_losses against the oracle's forward-mode derivatives
    (complex step) for a loss on both series: the squared distance of the
    moment loop from a target plus a soft maximum of the Joule power (the
    quench-onset term), along n, C_eps and a random Jc-factor direction."""
    from oracle.tangent import directional_derivatives
    from paper_2403_07666_b300.coil import Coil
    w = _loop_coil(thermal, transport, Y_eff)
    kw = {} if form == "fp64" else {"precision": "fp32", "format": "toeplitz_tc"}
    target = _oracle_moments(w, f=w.jc_factor * 1.05, n=27.0)
    with Coil.from_workload(w, rtol=1e-11, **kw) as c:
        s0 = c.save_state()
        c.step(K, w.drive)
        d = c.diag(0, K)
        m, P = d[:, 3], d[:, 4]
        c.load_state(s0)
        scale = 0.05 * np.max(P)
        _, dLdP = _soft_max_power(P, scale)
        dLdm = 2.0 * (m - target)
        gf, gn, gc = c.adjoint_losses(K, w.drive, dLdm, dLdP, ckpt_every=9)
        # the moment-only call equals coil_adjoint
        c.load_state(s0)
        gf_m, gn_m, gc_m = c.adjoint_losses(K, w.drive, dLdm, None, ckpt_every=9)
        c.load_state(s0)
        gf_a, gn_a, gc_a = c.adjoint(K, w.drive, dLdm, ckpt_every=9)
    assert np.array_equal(gf_m, gf_a) and gn_m == gn_a and gc_m == gc_a
    rng = np.random.default_rng(6)
    v = rng.standard_normal(w.n_elem)
    for vkw, ad in (({"v_n": 1.0}, gn), ({"v_C": 1.0}, gc), ({"v_f": v}, float(np.sum(gf * v)))):
        _, _, dm, dP = directional_derivatives(w, K, **vkw)
        tl = float(np.sum(dLdm * dm) + np.sum(dLdP * dP))
        assert abs(ad - tl) <= tol * abs(tl), (vkw.keys(), ad, tl)
    # the power term matters: dropping it changes the gradient
    assert abs(gn - gn_m) > 1e-3 * abs(gn)


def test_series_autograd_function_backward():
    import torch
    from paper_2403_07666_b300.autograd import CoilSeries
    from paper_2403_07666_b300.coil import Coil
    w = _loop_coil(1, 0)
    with Coil.from_workload(w, rtol=1e-11) as c, Coil.from_workload(w, rtol=1e-11) as c2:
        f = torch.tensor(w.jc_factor, dtype=torch.float64, requires_grad=True)
        n = torch.tensor(30.0, dtype=torch.float64, requires_grad=True)
        ce = torch.tensor(900.0, dtype=torch.float64, requires_grad=True)
        m, P = CoilSeries.apply(c, w.drive, K, 10, f, n, ce)
        scale = 0.05 * float(P.max())
        L = torch.sum(m ** 2) * 1e6 + scale * torch.logsumexp(P / scale, 0)
        L.backward()
        s0 = c2.save_state()
        c2.step(K, w.drive)
        d = c2.diag(0, K)
        c2.load_state(s0)
        _, dLdP = _soft_max_power(d[:, 4], scale)
        gf, gn, gc = c2.adjoint_losses(K, w.drive, 2e6 * d[:, 3], dLdP, ckpt_every=10)
    assert np.allclose(f.grad.numpy(), gf, rtol=1e-10, atol=1e-300)
    assert abs(n.grad.item() - gn) <= 1e-10 * abs(gn)
    assert abs(ce.grad.item() - gc) <= 1e-10 * abs(gc)
