"""GPU: batched cubes of uneven fold and azimuth coverage (one plan, one
persistent launch per stage), per-cube sparse solves and the autotuner,
against the oracle run cube by cube on the batch's shared time plan."""
import numpy as np
import pytest
import torch

import oracle
from oracle import fista, ops
from paper_2505_00387_gb300 import synthetic as syn

from gpu_util import dev, host, rel

pytestmark = pytest.mark.gpu

TOL_OP = 1e-4
TOL_SOLVE = 1e-3


def small_batch(cubes=(5, 17, 40), fold=150):
    cs = syn.cube_batch(ncube=len(cubes), cubes=list(cubes))
    for c in cs:                 # smaller folds keep the oracle quick
        c.hx, c.hy = c.hx[:fold], c.hy[:fold]
        c.d = c.d[:, :fold]
    r2max = max(float(np.max(c.hx ** 2 + c.hy ** 2)) for c in cs)
    ops_ = [oracle.make_plan(**c.geom_kwargs(), r2max=r2max) for c in cs]
    return cs, ops_


def split(x, sizes):
    out, o = [], 0
    for n in sizes:
        out.append(x[o:o + n])
        o += n
    return out


@pytest.fixture(scope="module")
def batch():
    from paper_2505_00387_gb300.plan import AahrtPlan
    cs, ops_ = small_batch()
    gp = AahrtPlan.batched(cs)
    return cs, ops_, gp


def test_per_cube_solve_matches_oracle(batch):
    cs, ops_, gp = batch
    gam, lam = [], []
    for c, p in zip(cs, ops_):
        gam.append(float(np.float32(0.95 / fista.power_sigma2(p, c.d))))
        lam.append(float(np.float32(0.05 * np.abs(ops.adjoint(p, c.d)).max())))
    cg, cl = np.array(gam), np.array(lam)
    d = dev(np.concatenate([c.d.ravel() for c in cs]))
    m, info = gp.sparse_solve(d, 0.0, 20, per_cube=True, cube_gamma=cg, cube_lambda=cl)
    mh = split(host(m), [c.ntau * c.nq * c.ntheta for c in cs])
    obj = 0.0
    for c, p, mg, g_, l_ in zip(cs, ops_, mh, gam, lam):
        ref = fista.solve(p, c.d, l_, 20, g_)
        assert rel(mg.reshape(ref.shape), ref) <= TOL_SOLVE
        obj += fista.objective(p, c.d, ref, l_)
    # the given values were used and handed back
    np.testing.assert_allclose(cg, gam, rtol=0, atol=0)
    assert abs(info.objective - obj) <= 1e-3 * obj


def test_per_cube_estimates_match_oracle(batch):
    cs, ops_, gp = batch
    cg = np.zeros(len(cs))
    cl = np.zeros(len(cs))
    d = dev(np.concatenate([c.d.ravel() for c in cs]))
    gp.sparse_solve(d, 0.0, 0, per_cube=True, lambda_rel=0.05, cube_gamma=cg, cube_lambda=cl)
    for c, p, g_, l_ in zip(cs, ops_, cg, cl):
        lam_ref = 0.05 * np.abs(ops.adjoint(p, c.d)).max()
        assert abs(l_ - lam_ref) <= 1e-4 * lam_ref
        gam_ref = 0.95 / fista.power_sigma2(p, c.d)
        assert abs(g_ - gam_ref) <= 1e-3 * gam_ref


def test_per_cube_graph_and_eager_agree(batch):
    cs, ops_, gp = batch
    d = dev(np.concatenate([c.d.ravel() for c in cs]))
    cg = np.zeros(len(cs))
    cl = np.zeros(len(cs))
    m1, _ = gp.sparse_solve(d, 0.0, 10, per_cube=True, lambda_rel=0.05, cube_gamma=cg,
                            cube_lambda=cl, use_graph=True, want_info=False)
    m2, _ = gp.sparse_solve(d, 0.0, 10, per_cube=True, cube_gamma=cg.copy(),
                            cube_lambda=cl.copy(), use_graph=False, want_info=False)
    torch.cuda.synchronize()
    assert torch.equal(m1, m2)


@pytest.mark.parametrize("pairs", [1, 4])
def test_time_pairs_do_not_change_results(batch, pairs):
    from paper_2505_00387_gb300.plan import AahrtPlan
    cs, ops_, gp = batch
    gq = AahrtPlan.batched(cs, time_pairs=pairs)
    assert gq.info.time_pairs == pairs
    rng = np.random.default_rng(70)
    m = dev(rng.standard_normal(gp.model_len))
    d = dev(rng.standard_normal(gp.data_len))
    assert torch.equal(gp.forward(m), gq.forward(m))
    assert torch.equal(gp.adjoint(d), gq.adjoint(d))


def test_autotuned_plan_is_correct(batch):
    from paper_2505_00387_gb300.plan import AahrtPlan
    cs, ops_, _ = batch
    gt = AahrtPlan.batched(cs, autotune=True)
    inf = gt.info
    assert inf.autotuned == 1 and inf.tune_ms > 0.0
    assert 5 <= inf.spread_width <= 12 and inf.time_pairs in (1, 2, 4, 8)
    assert 1 <= inf.theta_group <= cs[0].ntheta
    rng = np.random.default_rng(71)
    ms = [rng.standard_normal((c.ntau, c.nq, c.ntheta)) for c in cs]
    dg = host(gt.forward(dev(np.concatenate([m.ravel() for m in ms]))))
    for c, p, m, dgi in zip(cs, ops_, ms, split(dg, [c.nt * c.ntr for c in cs])):
        assert rel(dgi.reshape(c.nt, c.ntr), ops.forward(p, m)) < TOL_OP
    # explicit choices are kept
    gk = AahrtPlan.batched(cs, autotune=True, theta_group=6, spread_width=9)
    assert gk.info.theta_group == 6 and gk.info.spread_width == 9


@pytest.mark.slow
def test_batch512_sampled_parity():
    """The full 512-cube batch (fold 200-3000, sectors of 90-360 degrees, 64 q x
    24 azimuths): one autotuned plan; forward, adjoint and a 50-iteration
    per-cube FISTA solve checked on sampled cubes against the oracle."""
    from paper_2505_00387_gb300.plan import AahrtPlan
    cs = syn.cube_batch()
    gp = AahrtPlan.batched(cs, autotune=True)
    r2max = max(float(np.max(c.hx ** 2 + c.hy ** 2)) for c in cs)
    folds = np.array([c.ntr for c in cs])
    order = np.argsort(folds)
    sample = [int(order[0]), int(order[len(order) // 2])]   # smallest and median fold
    rng = np.random.default_rng(72)
    m = rng.standard_normal(gp.model_len)
    dgl = host(gp.forward(dev(m)))
    mgl = host(gp.adjoint(dev(np.concatenate([c.d.ravel() for c in cs]))))
    dsz = [c.nt * c.ntr for c in cs]
    msz = [c.ntau * c.nq * c.ntheta for c in cs]
    dsp, msp, mrs = split(dgl, dsz), split(mgl, msz), split(m, msz)
    ops_ = {i: oracle.make_plan(**cs[i].geom_kwargs(), r2max=r2max) for i in sample}
    for i in sample:
        c, p = cs[i], ops_[i]
        assert rel(dsp[i].reshape(c.nt, c.ntr), ops.forward(p, mrs[i].reshape(c.ntau, c.nq, c.ntheta))) < TOL_OP
        assert rel(msp[i].reshape(c.ntau, c.nq, c.ntheta), ops.adjoint(p, c.d)) < TOL_OP
    # per-cube solve; the sampled cubes get the oracle's step and threshold
    cg = np.zeros(len(cs))
    cl = np.zeros(len(cs))
    lam_ref = {}
    for i in sample:
        c, p = cs[i], ops_[i]
        cg[i] = float(np.float32(0.95 / fista.power_sigma2(p, c.d)))
        lam_ref[i] = float(np.float32(0.05 * np.abs(ops.adjoint(p, c.d)).max()))
    # lambda_rel would override the given lambdas: give every cube its own
    # lambda from a first estimate, then the oracle's for the sampled cubes
    est_g, est_l = np.zeros(len(cs)), np.zeros(len(cs))
    d = dev(np.concatenate([c.d.ravel() for c in cs]))
    gp.sparse_solve(d, 0.0, 0, per_cube=True, lambda_rel=0.05, cube_gamma=est_g,
                    cube_lambda=est_l, want_info=False)
    for i in sample:
        cl_i = lam_ref[i]
        assert abs(est_l[i] - cl_i) <= 1e-4 * cl_i
        est_l[i] = cl_i
        est_g[i] = cg[i]
    m_sol, info = gp.sparse_solve(d, 0.0, 50, per_cube=True, cube_gamma=est_g,
                                  cube_lambda=est_l)
    ms = split(host(m_sol), msz)
    for i in sample:
        c, p = cs[i], ops_[i]
        ref = fista.solve(p, c.d, est_l[i], 50, est_g[i])
        assert rel(ms[i].reshape(ref.shape), ref) <= TOL_SOLVE


def test_single_cube_on_the_batch_time_plan():
    """A cube planned alone with the batch's largest squared offset (opts
    r2max) gets the batch's stretched-time plan and so the same operator:
    its forward and adjoint equal the batched plan's on that cube (the
    per-cube form of the same work).  An r2max below the
    cube's own offsets is refused."""
    from paper_2505_00387_gb300 import _lib as L
    from paper_2505_00387_gb300.plan import AahrtPlan
    cs, _ = small_batch()
    r2max = max(float(np.max(c.hx ** 2 + c.hy ** 2)) for c in cs)
    bp = AahrtPlan.batched(cs)
    i = int(np.argmin([float(np.max(x.hx ** 2 + x.hy ** 2)) for x in cs]))
    c = cs[i]
    assert float(np.max(c.hx ** 2 + c.hy ** 2)) < r2max
    sp = AahrtPlan(**c.geom_kwargs(), r2max=r2max)
    for f in ("nfft", "ns", "nbins", "spread_width"):
        assert getattr(sp.info, f) == getattr(bp.info, f), f
    assert sp.info.ds == bp.info.ds
    own = AahrtPlan(**c.geom_kwargs())
    assert own.info.rho < sp.info.rho
    rng = np.random.default_rng(71)
    ms = [rng.standard_normal((x.ntau, x.nq, x.ntheta)) for x in cs]
    ds = [rng.standard_normal((x.nt, x.ntr)) for x in cs]
    dg = split(host(bp.forward(dev(np.concatenate([m.ravel() for m in ms])))),
               [x.nt * x.ntr for x in cs])
    mg = split(host(bp.adjoint(dev(np.concatenate([d.ravel() for d in ds])))),
               [m.size for m in ms])
    assert rel(host(sp.forward(dev(ms[i]))), dg[i]) < 1e-6
    assert rel(host(sp.adjoint(dev(ds[i]))), mg[i]) < 1e-6
    with pytest.raises(L.AahrtError) as e:
        AahrtPlan(**c.geom_kwargs(), r2max=0.5 * float(np.max(c.hx ** 2 + c.hy ** 2)))
    assert e.value.status == L.AAHRT_ERR_INVALID_ARG
