"""GPU: the q-moment velocity pick (eq. vel_est) through the C ABI against
the oracle, for single, batched and tensor-core (gather-fastest) plans, and
end to end: a GPU sparse solve of small-cube data picked at each isolated
event tracks the generator's elliptical curvature."""
import numpy as np
import pytest

import oracle
from oracle import ops, pick
from paper_2505_00387_gb300 import synthetic as syn

from gpu_util import dev, gpu_plan, host, oracle_plan

pytestmark = pytest.mark.gpu


def check(qg, wg, qo, wo):
    np.testing.assert_allclose(wg, wo, rtol=2e-6, atol=1e-6 * wo.max())
    ok = wo > 1e-3 * wo.max()
    np.testing.assert_allclose(qg[ok], qo[ok], rtol=1e-5, atol=0)


def test_pick_matches_oracle_single_and_batched():
    g = syn.small_cube()
    op = oracle_plan(g)
    gp = gpu_plan(g)
    rng = np.random.default_rng(100)
    m = rng.standard_normal(g.m.shape) * (rng.random(g.m.shape) < 0.3)
    qg, wg = gp.pick_velocity(dev(m))
    qo, wo = pick.pick(op, m)
    check(host(qg, qo.shape), host(wg, wo.shape), qo, wo)

    from paper_2505_00387_gb300.plan import AahrtPlan
    cubes = syn.cube_batch(ncube=2, cubes=[3, 9])
    gb = AahrtPlan.batched(cubes)
    ms = [rng.standard_normal((c.ntau, c.nq, c.ntheta)) for c in cubes]
    qg, wg = gb.pick_velocity(dev(np.concatenate([x.ravel() for x in ms])))
    n = cubes[0].ntau * cubes[0].ntheta
    for i, (c, x) in enumerate(zip(cubes, ms)):
        qo, wo = pick.pick(oracle.make_plan(**c.geom_kwargs()), x)
        check(host(qg)[i * n:(i + 1) * n].reshape(qo.shape),
              host(wg)[i * n:(i + 1) * n].reshape(wo.shape), qo, wo)


def test_pick_tensorcore_layout():
    g = syn.small_cube()
    op = oracle_plan(g)
    G = 3
    gp = gpu_plan(g, ngather=G, precision="split_bf16")
    rng = np.random.default_rng(101)
    ms = [rng.standard_normal(g.m.shape) for _ in range(G)]
    qg, wg = gp.pick_velocity(dev(np.stack(ms, axis=-1)))
    qg = host(qg).reshape(g.ntau, g.ntheta, G)
    wg = host(wg).reshape(g.ntau, g.ntheta, G)
    for i in range(G):
        qo, wo = pick.pick(op, ms[i])
        check(qg[..., i], wg[..., i], qo, wo)


def test_pick_after_gpu_solve_tracks_the_ellipse():
    g = syn.small_cube()
    op = oracle_plan(g)
    gp = gpu_plan(g)
    d = ops.forward(op, g.m)
    m, _ = gp.sparse_solve(dev(d), 0.0, 60, lambda_rel=0.05, want_info=False)
    qg, _ = gp.pick_velocity(m)
    qg = host(qg, (g.ntau, g.ntheta))
    th = np.arange(g.ntheta) * np.pi / g.ntheta
    checked = 0
    for sp in g.info["spikes"]:
        if any(abs(o["tau"] - sp["tau"]) < 0.06 for o in g.info["spikes"] if o is not sp):
            continue
        i = int(round(sp["tau"] / g.dt))
        qe = np.clip(syn.ellipse_q(th, sp["v"], sp["v"] / 1.1, sp["axis"]), op.q[0], op.q[-1])
        assert np.max(np.abs(qg[i] - qe)) <= 0.5 * g.dq
        checked += 1
    assert checked >= 2
