"""GPU path (through the C ABI) against the FP64 oracle on the same seeded
inputs.  Tolerances: each operator application <= 1e-4 relative L2, FISTA
output after a fixed number of iterations <= 1e-3, FP32 dot-product
(adjoint) test <= 1e-6 relative."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import fista, ops
from paper_2505_00387_gb300 import synthetic as syn

from gpu_util import dev, dot_rel_conditioned, gpu_plan, host, oracle_H, oracle_plan, rel

pytestmark = pytest.mark.gpu

TOL_OP = 1e-4
TOL_FISTA = 1e-3
TOL_DOT = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_00387_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def small_case():
    g = syn.small_cube()
    p = oracle_plan(g)
    return g, p, gpu_plan(g)


def test_plan_matches_oracle_sampling(small_case):
    g, p, gp = small_case
    assert gp.info.nfft == p.nfft and gp.info.ns == p.ns and gp.info.nbins == p.nbins
    assert abs(gp.info.ds - p.ds) <= 1e-12 * p.ds


def test_stages_small_cube(small_case):
    g, p, gp = small_case
    rng = np.random.default_rng(20)
    m = g.m
    nb = p.nbins
    # stage 0: X = F S m
    X = host(gp.apply_stage(0, dev(m)), (nb, p.nq, p.ntheta))
    Xo = ops.rfft_bins(p, ops.stretch(p, m.reshape(p.ntau, -1))).reshape(nb, p.nq, p.ntheta)
    assert rel(X, Xo) < 2e-6
    # stage 1: Y = P X / nfft on the oracle's X
    Xc = torch.from_numpy(Xo.astype(np.complex64).ravel()).cuda()
    Y = host(gp.apply_stage(1, Xc), (nb, p.ntr))
    Yo = ops.slice_forward(p, Xo) / p.nfft
    assert rel(Y, Yo) < 1e-5
    # stage 2: d = U H Y
    Yc = torch.from_numpy(Yo.astype(np.complex64).ravel()).cuda()
    d = host(gp.apply_stage(2, Yc), (p.nt, p.ntr))
    do = ops.unstretch(p, oracle_H(p, Yo))
    assert rel(d, do) < 2e-6
    # stage 3: Y = F U^T d
    dr = rng.standard_normal((p.nt, p.ntr))
    Y3 = host(gp.apply_stage(3, dev(dr)), (nb, p.ntr))
    Y3o = ops.rfft_bins(p, ops.unstretch_T(p, dr))
    assert rel(Y3, Y3o) < 2e-6
    # stage 4: X = P^H Y / nfft
    X4 = host(gp.apply_stage(4, torch.from_numpy(Y3o.astype(np.complex64).ravel()).cuda()),
              (nb, p.nq, p.ntheta))
    X4o = ops.slice_adjoint(p, Y3o) / p.nfft
    assert rel(X4, X4o) < 1e-5
    # stage 5: m = S^T H X
    m5 = host(gp.apply_stage(5, torch.from_numpy(X4o.astype(np.complex64).ravel()).cuda()),
              (p.ntau, p.nq, p.ntheta))
    m5o = ops.stretch_T(p, oracle_H(p, X4o.reshape(nb, -1))).reshape(p.ntau, p.nq, p.ntheta)
    assert rel(m5, m5o) < 2e-6


def test_forward_adjoint_small_cube(small_case):
    g, p, gp = small_case
    d = host(gp.forward(dev(g.m)), (p.nt, p.ntr))
    assert rel(d, ops.forward(p, g.m)) < TOL_OP
    rng = np.random.default_rng(21)
    dr = rng.standard_normal((p.nt, p.ntr))
    m = host(gp.adjoint(dev(dr)), (p.ntau, p.nq, p.ntheta))
    assert rel(m, ops.adjoint(p, dr)) < TOL_OP


def _dot_test(gp, p, seed):
    """Relative FP32 dot-test error on a well-conditioned pair (d = L m by
    the oracle plan p, plus noise)."""
    return dot_rel_conditioned(
        gp, lambda m: ops.forward(p, m.reshape(p.ntau, p.nq, p.ntheta)), seed)


def test_dot_product_small_cube(small_case):
    g, p, gp = small_case
    assert _dot_test(gp, p, 22) < TOL_DOT


def test_fista_small_cube(small_case):
    g, p, gp = small_case
    d = ops.forward(p, g.m)
    lam = 0.05 * float(np.abs(ops.adjoint(p, d)).max())
    gamma = 0.95 / fista.power_sigma2(p, d, iters=30)
    mo = fista.solve(p, d, lam, 20, gamma)
    for graph in (True, False):
        mg, info = gp.sparse_solve(dev(d), lam, 20, gamma=gamma, use_graph=graph)
        assert rel(host(mg, mo.shape), mo) < TOL_FISTA
        assert info.iters == 20
        r = np.linalg.norm(d - ops.forward(p, mo))
        assert abs(info.resid_norm - r) / r < 1e-3
    mi = fista.solve(p, d, lam, 10, gamma, momentum=False)
    mg, _ = gp.sparse_solve(dev(d), lam, 10, gamma=gamma, ista=True)
    assert rel(host(mg, mi.shape), mi) < TOL_FISTA


def test_solver_estimates_gamma_and_lambda(small_case):
    """gamma from the device power iteration and lambda = 0.05 max|L^T d|."""
    g, p, gp = small_case
    d = ops.forward(p, g.m)
    lam = 0.05 * float(np.abs(ops.adjoint(p, d)).max())
    sig2 = fista.power_sigma2(p, d, iters=30)
    _, info = gp.sparse_solve(dev(d), 0.0, 2, lambda_rel=0.05)
    assert abs(getattr(info, "lambda") - lam) / lam < 1e-4
    assert abs(info.gamma - 0.95 / sig2) / (0.95 / sig2) < 1e-3


# ----------------------------------------------------------- ragged cases
def _ragged_gather(nt=300, ntr=333, nq=37, nth=5, seed=30, q0=None):
    rng = np.random.default_rng(seed)
    hx, hy = syn.disc_offsets(rng, ntr, 2500.0)
    a, b = syn.q_axis(nq)
    if q0 is not None:
        a = q0
    return syn.Gather(nt, 0.004, nt + 7, nq, a, b, nth, hx, hy)


@pytest.mark.parametrize("interp,tg,w", [("keys", 0, 7), ("linear", 2, 6), ("keys", 2, 9),
                                         ("keys", 3, 5)])
def test_ragged_multigroup(interp, tg, w):
    g = _ragged_gather()
    p = oracle_plan(g, interp=interp)
    gp = gpu_plan(g, interp=interp, theta_group=tg, spread_width=w)
    if tg:
        assert gp.info.theta_group == tg
    rng = np.random.default_rng(31)
    m = rng.standard_normal((g.ntau, g.nq, g.ntheta))
    d = rng.standard_normal((g.nt, g.ntr))
    tol = TOL_OP if w >= 6 else 5e-4
    assert rel(host(gp.forward(dev(m)), (g.nt, g.ntr)), ops.forward(p, m)) < tol
    assert rel(host(gp.adjoint(dev(d)), m.shape), ops.adjoint(p, d)) < tol
    assert _dot_test(gp, p, 32) < TOL_DOT


@pytest.mark.parametrize("case", ["one_azimuth", "one_curvature", "zero_offset",
                                  "negative_q", "single_slice", "short", "fmax"])
def test_edge_cases(case):
    rng = np.random.default_rng(40)
    kw = {}
    if case == "one_azimuth":
        g = _ragged_gather(nth=1, ntr=50)
    elif case == "one_curvature":
        g = _ragged_gather(nq=1, ntr=40)
    elif case == "zero_offset":
        g = _ragged_gather(ntr=41)
        g.hx[:3] = 0.0
        g.hy[:3] = 0.0
    elif case == "negative_q":
        g = _ragged_gather(nq=24, q0=-2e-7)
    elif case == "single_slice":
        g = _ragged_gather(ntr=30)
        g.hy[:] = 0.0
        g.hx[:] = np.abs(g.hx) + 10.0
    elif case == "short":
        g = _ragged_gather(nt=8, ntr=5, nq=3, nth=2)
        g.ntau, g.dt = 8, 0.05
        g.hx, g.hy = g.hx * 0.2, g.hy * 0.2
    else:
        g = _ragged_gather(ntr=60)
        kw = dict(fmax=30.0)
    p = oracle_plan(g, **kw)
    gp = gpu_plan(g, **kw)
    assert gp.info.nbins == p.nbins
    m = rng.standard_normal((g.ntau, g.nq, g.ntheta))
    d = rng.standard_normal((g.nt, g.ntr))
    assert rel(host(gp.forward(dev(m)), (g.nt, g.ntr)), ops.forward(p, m)) < TOL_OP
    assert rel(host(gp.adjoint(dev(d)), m.shape), ops.adjoint(p, d)) < TOL_OP
    assert _dot_test(gp, p, 41) < TOL_DOT


# q grids of nos = 32, 128 and 512 points (the adjoint's inverse q-FFT as a
# first and a last step, or with middle steps); one azimuth group with the
# wrap from the last slice to slice 0, or groups of 2 slices with edge traces;
# up to 2600 traces (ten per thread) in one work item
@pytest.mark.parametrize("nq,ntr,nth,tg", [(9, 700, 4, 0), (37, 2600, 3, 0), (37, 2600, 6, 2),
                                           (150, 400, 4, 2)])
def test_adjoint_grid_sizes_and_repeatability(nq, ntr, nth, tg):
    """Adjoint parity across q-grid sizes and group layouts, and bitwise
    repeatable output: the spread's shared-memory integer atomics land in
    whatever order the warps reach them, and the sums must not depend on it."""
    g = _ragged_gather(ntr=ntr, nq=nq, nth=nth, seed=33)
    p = oracle_plan(g)
    gp = gpu_plan(g, theta_group=tg)
    rng = np.random.default_rng(34)
    d = rng.standard_normal((g.nt, g.ntr))
    shape = (g.ntau, g.nq, g.ntheta)
    m1 = host(gp.adjoint(dev(d)), shape)
    m2 = host(gp.adjoint(dev(d)), shape)
    np.testing.assert_array_equal(m1, m2)
    assert rel(m1, ops.adjoint(p, d)) < TOL_OP
    assert _dot_test(gp, p, 35) < TOL_DOT


def test_plan_refuses_oversized_frame():
    from paper_2505_00387_gb300 import _lib as L
    g = _ragged_gather(nt=8, ntr=5, nq=3, nth=2)
    g.ntau = 8
    with pytest.raises(L.AahrtError) as e:
        gpu_plan(g)
    assert e.value.status == L.AAHRT_ERR_UNSUPPORTED
    assert "nt = 8" in str(e.value)


# ---------------------------------------------------- batches and gathers
def test_batched_cubes_match_oracle():
    cubes = syn.cube_batch(ncube=3, cubes=[5, 17, 40])
    for c in cubes:          # smaller folds keep the oracle quick
        c.hx, c.hy = c.hx[:150], c.hy[:150]
        c.d = c.d[:, :150]
    from paper_2505_00387_gb300.plan import AahrtPlan
    gp = AahrtPlan.batched(cubes)
    r2max = max(float(np.max(c.hx ** 2 + c.hy ** 2)) for c in cubes)
    rng = np.random.default_rng(50)
    ms = [rng.standard_normal((c.ntau, c.nq, c.ntheta)) for c in cubes]
    ds = [rng.standard_normal((c.nt, c.ntr)) for c in cubes]
    dg = host(gp.forward(dev(np.concatenate([m.ravel() for m in ms]))))
    mg = host(gp.adjoint(dev(np.concatenate([d.ravel() for d in ds]))))
    off_d = off_m = 0
    for c, m, d in zip(cubes, ms, ds):
        p = oracle.make_plan(**c.geom_kwargs(), r2max=r2max)
        n_d, n_m = c.nt * c.ntr, m.size
        assert rel(dg[off_d:off_d + n_d].reshape(c.nt, c.ntr), ops.forward(p, m)) < TOL_OP
        assert rel(mg[off_m:off_m + n_m].reshape(m.shape), ops.adjoint(p, d)) < TOL_OP
        off_d += n_d
        off_m += n_m
    plans = [oracle.make_plan(**c.geom_kwargs(), r2max=r2max) for c in cubes]

    def fwd_all(mflat):
        out, off = [], 0
        for c, pc in zip(cubes, plans):
            n = c.ntau * c.nq * c.ntheta
            out.append(ops.forward(pc, mflat[off:off + n].reshape(c.ntau, c.nq, c.ntheta)).ravel())
            off += n
        return np.concatenate(out)

    assert dot_rel_conditioned(gp, fwd_all, 51) < TOL_DOT


def test_shared_geometry_gathers_match_single():
    g = _ragged_gather(ntr=120)
    G = 3
    g1 = gpu_plan(g)
    gG = gpu_plan(g, ngather=G)
    assert gG.model_len == G * g1.model_len and gG.data_len == G * g1.data_len
    rng = np.random.default_rng(60)
    m = rng.standard_normal((G, g1.model_len))
    dG = host(gG.forward(dev(m)))
    for i in range(G):
        di = host(g1.forward(dev(m[i])))
        np.testing.assert_array_equal(dG[i * g1.data_len:(i + 1) * g1.data_len], di)


# ------------------------------------------------------------- API errors
def test_api_rejects_bad_pointers(small_case):
    from paper_2505_00387_gb300 import _lib as L
    g, p, gp = small_case
    m = torch.zeros(gp.model_len + 8, device="cuda")
    d = torch.zeros(gp.data_len, device="cuda")
    with pytest.raises(L.AahrtError) as e:
        L.aahrt_forward(gp.handle, m.data_ptr() + 4, d.data_ptr())
    assert e.value.status == L.AAHRT_ERR_INVALID_ARG
    # host buffers are staged through the plan and give the device result
    hm = np.random.default_rng(80).standard_normal(gp.model_len).astype(np.float32)
    hd = np.zeros(gp.data_len, np.float32)
    L.aahrt_forward(gp.handle, hm.ctypes.data, hd.ctypes.data)
    torch.cuda.synchronize()
    want = host(gp.forward(torch.from_numpy(hm).cuda()))
    np.testing.assert_array_equal(hd, want.astype(np.float32))
    with pytest.raises(L.AahrtError) as e:
        L.aahrt_forward(gp.handle, hm.ctypes.data + 1, d.data_ptr())
    assert e.value.status == L.AAHRT_ERR_INVALID_ARG
    with pytest.raises(L.AahrtError) as e:
        L.aahrt_apply_stage(gp.handle, 9, m.data_ptr(), d.data_ptr())
    assert e.value.status == L.AAHRT_ERR_INVALID_ARG
    # the context still works
    gp.forward(m[:gp.model_len].contiguous(), d)
    torch.cuda.synchronize()


def test_profiling_counts_stages(small_case):
    g, p, gp = small_case
    gp.set_profiling(True)
    d = gp.forward(dev(g.m))
    gp.adjoint(d)
    t, n = gp.stage_times()
    gp.set_profiling(False)
    assert n[:6] == [1, 1, 1, 1, 1, 1]
    assert all(x > 0 for x in t[:6])


# ------------------------------------------------- paper-scale gather
@pytest.fixture(scope="module")
def paper_case():
    g = syn.paper_gather()
    return g, oracle_plan(g), gpu_plan(g)


def test_paper_gather_sampled_forward_adjoint(paper_case):
    g, p, gp = paper_case
    rng = np.random.default_rng(70)
    m = rng.standard_normal((g.ntau, g.nq, g.ntheta)).astype(np.float32).astype(np.float64)
    dg = host(gp.forward(dev(m)), (g.nt, g.ntr))
    traces = [0, 7, 999, 1500, g.ntr - 1]
    assert rel(dg[:, traces], ops.forward_traces(p, m, traces)) < TOL_OP
    mg = host(gp.adjoint(dev(g.d)), (g.ntau, g.nq, g.ntheta))
    slices = [0, 17, g.ntheta - 1]
    assert rel(mg[:, :, slices], ops.adjoint_slices(p, g.d, slices)) < TOL_OP


def test_paper_gather_dot_product(paper_case):
    g, p, gp = paper_case
    assert _dot_test(gp, p, 71) < TOL_DOT


def test_paper_gather_fista_few_iterations(paper_case):
    g, p, gp = paper_case
    d = g.d
    lam = 0.05 * float(np.abs(ops.adjoint(p, d)).max())
    gamma = 0.9 / fista.power_sigma2(p, d, iters=4)
    mo = fista.solve(p, d, lam, 3, gamma)
    mg, _ = gp.sparse_solve(dev(d), lam, 3, gamma=gamma)
    assert rel(host(mg, mo.shape), mo) < TOL_FISTA


@pytest.mark.slow
def test_paper_gather_fista_100_iterations(paper_case):
    """The paper-scale gather's full solve: 100 FISTA iterations through
    aahrt_sparse_solve against the oracle's solve with the oracle's step
    (0.95 / sigma^2 from 30 power iterations) and threshold
    (lambda = 0.05 max|L^T d|), on the whole model cube."""
    g, p, gp = paper_case
    d = g.d
    lam = 0.05 * float(np.abs(ops.adjoint(p, d)).max())
    gamma = 0.95 / fista.power_sigma2(p, d, iters=30)
    mo = fista.solve(p, d, lam, 100, gamma)
    for graph in (True, False):
        mg, info = gp.sparse_solve(dev(d), lam, 100, gamma=gamma, use_graph=graph)
        assert info.iters == 100
        err = rel(host(mg, mo.shape), mo)
        assert err < TOL_FISTA, f"graph={graph}: rel {err:.3e}"
