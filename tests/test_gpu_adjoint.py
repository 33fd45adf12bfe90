"""The moments adjoint on the GPU (vt_moments_adjoint, VoronoiMoments, lloyd)
against the oracle adjoint and the closed forms that pin it.

Tolerances: FP64 tessellation -> 1e-9 relative to the largest gradient
component (face integrals of the same cells, different quadrature order);
FP32 tessellation -> 1e-4 (vertices carry float32 round-off).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2412_04514_gb300 as vt
from oracle import adjoint as oadj
from paper_2412_04514_gb300 import workloads as W

pytestmark = pytest.mark.gpu

EMIT = ("vol", "cen", "m2", "geom")


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.fixture(scope="module")
def small():
    p = W.uniform(4096, 0)
    rng = np.random.default_rng(8)
    g = rng.standard_normal(len(p)), rng.standard_normal((len(p), 3)), rng.standard_normal(len(p))
    return p, g, oadj.moments_adjoint(p, *g)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("fp32", 1e-4)])
def test_adjoint_matches_oracle(small, prec, tol):
    p, (gV, gC, gM), want = small
    d = dev(p)
    cells = vt.tessellate(d, vt.Params(precision=prec, emit=EMIT))
    got = vt.moments_adjoint(d, cells, dev(gV), dev(gC), dev(gM), precision=prec).cpu().numpy()
    scale = np.abs(want).max()
    assert np.abs(got - want).max() <= tol * scale


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("fp32", 1e-4)])
def test_lloyd_identity_and_conservation_on_the_bench_cloud(prec, tol):
    p = W.mixed(1 << 20, 1)
    d = dev(p)
    cells = vt.tessellate(d, vt.Params(precision=prec, emit=EMIT))
    n = len(p)
    ones = torch.ones(n, dtype=torch.float64, device="cuda")
    g = vt.moments_adjoint(d, cells, gM=ones, precision=prec)
    want = 2 * cells.vol[:, None] * (d.double() - cells.cen)
    scale = want.abs().max()
    assert float((g - want).abs().max()) <= tol * float(scale)
    g = vt.moments_adjoint(d, cells, gV=ones, precision=prec)  # total volume does not move
    assert float(g.abs().max()) <= tol * float(cells.vol.max()) ** (2 / 3)


def test_adjoint_matches_finite_differences_of_the_gpu_forward():
    n = 256
    p = W.uniform(n, 5)
    rng = np.random.default_rng(55)
    gV, gC, gM = rng.standard_normal(n), rng.standard_normal((n, 3)), rng.standard_normal(n)
    prm = vt.Params(precision="fp64", emit=EMIT)
    d = dev(p)
    cells = vt.tessellate(d, prm)
    g = vt.moments_adjoint(d, cells, dev(gV), dev(gC), dev(gM)).cpu().numpy()

    def loss(q):
        c = vt.tessellate(dev(q), prm)
        return float(np.sum(gV * c.vol.cpu().numpy()) + np.sum(gC * c.cen.cpu().numpy())
                     + np.sum(gM * c.m2.cpu().numpy()))

    def central(k, a, h):
        pp, pm = p.copy(), p.copy()
        pp[k, a] = np.float32(p[k, a] + h)
        pm[k, a] = np.float32(p[k, a] - h)
        return (loss(pp) - loss(pm)) / (np.float64(pp[k, a]) - np.float64(pm[k, a]))

    for k in rng.choice(n, 6, replace=False):
        for a in range(3):
            fd = (4 * central(k, a, 5e-5) - central(k, a, 1e-4)) / 3
            assert abs(fd - g[k, a]) <= 1e-6 * max(1.0, abs(g[k, a])), (k, a, fd, g[k, a])


def test_autograd_function_calls_the_adjoint(small):
    p, (gV, gC, gM), want = small
    q = dev(p).requires_grad_(True)
    vol, cen, m2 = vt.voronoi_moments(q, vt.Params(precision="fp64"))
    loss = (vol * dev(gV)).sum() + (cen * dev(gC)).sum() + (m2 * dev(gM)).sum()
    loss.backward()
    assert q.grad.dtype == torch.float32
    np.testing.assert_allclose(q.grad.cpu().numpy(), want.astype(np.float32), rtol=0,
                               atol=1e-5 * np.abs(want).max())


def test_lloyd_step_lands_on_the_oracle_centroids():
    p = W.uniform(2000, 9)
    out = vt.lloyd(dev(p), 2, vt.Params(precision="fp64")).cpu().numpy()
    q = p
    for _ in range(2):
        r = oracle.tessellate(q)
        q = r["cen"].astype(np.float32)
    np.testing.assert_allclose(out, q, rtol=0, atol=2e-7)


def test_lloyd_energy_decreases_and_resume_is_bit_identical(tmp_path):
    p = dev(W.uniform(20000, 4))
    energies = []
    full = vt.lloyd(p, 4, vt.Params(precision="fp32"), callback=lambda it, e: energies.append(e))
    assert all(b < a for a, b in zip(energies, energies[1:]))
    ck = str(tmp_path / "lloyd.pt")
    vt.lloyd(p, 2, vt.Params(precision="fp32"), checkpoint=ck, checkpoint_every=1)
    resumed = vt.lloyd(p, 4, vt.Params(precision="fp32"), checkpoint=ck, resume=True)
    assert torch.equal(full, resumed)


def test_lloyd_1m_uniform_50_iterations_decreases_the_energy():
    # the differentiation workload at full size: 1,048,576 uniform points, 50 iterations
    p = dev(W.uniform(1 << 20, 4))
    energies = []
    out = vt.lloyd(p, 50, vt.Params(precision="fp32"), callback=lambda it, e: energies.append(e))
    assert len(energies) == 50
    assert all(b <= a * (1 + 1e-9) for a, b in zip(energies, energies[1:]))
    assert energies[-1] < 0.97 * energies[0]
    assert bool(((out >= 0) & (out < 1)).all())


def test_lloyd_step_kernel_moves_wraps_and_clamps():
    # target points t = p - g / (2 V): inside, beyond hi and below lo (periodic
    # wrap by whole periods), and one that rounds onto hi
    p = np.array([[0.5, 0.5, 0.5], [0.9, 0.1, 0.2], [0.3, 0.4, 0.6]], np.float32)
    t = np.array([[0.25, 0.75, 0.125], [1.25, -0.5, 0.2], [1.0 - 1e-12, 0.4, 0.6]])
    vol = np.array([0.5, 2.0, 1.0])
    g = 2.0 * vol[:, None] * (p.astype(np.float64) - t)
    dp, dg, dv = dev(p), dev(g), dev(vol)
    walled = vt.lloyd_step(dp, dg, dv, vt.Params()).cpu().numpy()
    want = t.astype(np.float32)
    want[2, 0] = np.nextafter(np.float32(1), np.float32(0))  # rounds onto hi: the largest float below it
    want[1] = [1.25, -0.5, 0.2]  # a walled box does not wrap (the centroid never leaves it)
    assert np.array_equal(walled[[0, 2]], want[[0, 2]])
    per = vt.lloyd_step(dp, dg, dv, vt.Params(periodic=True)).cpu().numpy()
    assert np.array_equal(per[0], want[0])
    assert np.array_equal(per[1], np.array([0.25, 0.5, 0.2], np.float32))
    assert per[2, 0] == 0.0  # rounds onto hi: belongs at lo
