"""GPU: the split-BF16 tensor-core slice step (gathers on one geometry,
gather-fastest layout) against the oracle, gather by gather, and beside the
FP32 spreading path on the same inputs."""
import numpy as np
import pytest
import torch

import oracle
from oracle import ops
from paper_2505_00387_gb300 import synthetic as syn

from gpu_util import dev, gpu_plan, host, oracle_plan, rel

pytestmark = pytest.mark.gpu

TOL_OP = 1e-4          # operator application vs the FP64 oracle
TOL_DOT_TC = 5e-5      # split-bf16 forward and adjoint round differently


def interleave(xs):
    return np.stack(xs, axis=-1)


def run_pair(gp, ms, ds):
    d = host(gp.forward(dev(interleave(ms))))
    m = host(gp.adjoint(dev(interleave(ds))))
    gp.status()
    G = len(ms)
    return d.reshape(ds[0].shape + (G,)), m.reshape(ms[0].shape + (G,))


def ragged_geometry():
    """nq = 150 (two row tiles of q in the adjoint), 5 azimuth slices: slice 0
    holds more than 128 traces (two forward row tiles), slices 1 and 2 hold
    none, so slice 2 receives no contribution at all."""
    rng = np.random.default_rng(80)
    n1, n2 = 180, 60
    az1 = rng.uniform(0.0, 0.6, n1)            # slice 0 (width pi/5 = 0.63)
    az2 = rng.uniform(1.9, 3.1, n2)            # slices 3 and 4
    r = 1500.0 * np.sqrt(rng.uniform(0.05, 1.0, n1 + n2))
    az = np.concatenate([az1, az2]) + np.pi * rng.integers(0, 2, n1 + n2)
    hx, hy = r * np.cos(az), r * np.sin(az)
    q0, dq = syn.q_axis(150)
    return syn.Gather(192, 0.004, 192, 150, q0, dq, 5, hx, hy)


@pytest.mark.parametrize("case", ["small_cube", "ragged"])
@pytest.mark.parametrize("G", [4, 13])
def test_tensorcore_slice_matches_oracle(case, G):
    g = syn.small_cube() if case == "small_cube" else ragged_geometry()
    op = oracle_plan(g)
    gp = gpu_plan(g, ngather=G, precision="split_bf16")
    assert gp.info.precision == 1 and gp.info.ngather == G
    rng = np.random.default_rng(81)
    ms = [rng.standard_normal((g.ntau, g.nq, g.ntheta)) for _ in range(G)]
    ds = [rng.standard_normal((g.nt, g.ntr)) for _ in range(G)]
    dg, mg = run_pair(gp, ms, ds)
    for i in (0, G // 2, G - 1):
        assert rel(dg[..., i], ops.forward(op, ms[i])) < TOL_OP
        assert rel(mg[..., i], ops.adjoint(op, ds[i])) < TOL_OP
    # dot test over all gathers, at the split-bf16 rounding level
    lhs = float(np.sum(dg * interleave(ds)))
    rhs = float(np.sum(mg * interleave(ms)))
    assert abs(lhs - rhs) <= TOL_DOT_TC * (abs(lhs) + abs(rhs))


def test_tensorcore_matches_fp32_path_and_empty_slice():
    g = ragged_geometry()
    G = 3
    gt = gpu_plan(g, ngather=G, precision="split_bf16")
    gf = gpu_plan(g, ngather=G)
    rng = np.random.default_rng(82)
    ms = [rng.standard_normal((g.ntau, g.nq, g.ntheta)) for _ in range(G)]
    ds = [rng.standard_normal((g.nt, g.ntr)) for _ in range(G)]
    dt_, mt_ = run_pair(gt, ms, ds)
    df = host(gf.forward(dev(np.stack(ms)))).reshape((G,) + ds[0].shape)
    mf = host(gf.adjoint(dev(np.stack(ds)))).reshape((G,) + ms[0].shape)
    for i in range(G):
        assert rel(dt_[..., i], df[i]) < TOL_OP
        assert rel(mt_[..., i], mf[i]) < TOL_OP
    # slice 2 is touched by no trace: its adjoint spectrum is exactly zero
    op = oracle_plan(g)
    assert not (np.isin(op.j0, [2]) | np.isin(op.j1, [2])).any()
    X = gt.apply_stage(4, gt.apply_stage(3, dev(interleave(ds))))
    Xh = host(X).reshape(g.ntheta, gt.info.nbins, g.nq, G)      # slice-major spectra
    assert np.all(Xh[2] == 0) and np.any(Xh[1] != 0)


def test_tensorcore_rejects_unsupported():
    from paper_2505_00387_gb300._lib import AahrtError
    g = syn.small_cube()
    with pytest.raises(AahrtError):
        gpu_plan(g, ngather=65, precision="split_bf16")


@pytest.mark.slow
def test_shared_geometry_64_gathers_sampled():
    """64 gathers on one 8000-trace geometry (nt = 2048 at 2 ms, 200 q x 72
    azimuths): both slice paths, forward on sampled traces and adjoint on
    sampled azimuth slices of two gathers, against the oracle."""
    geo, _ = syn.shared_batch(gathers=[])
    G = 64
    op = oracle_plan(geo)
    rng = np.random.default_rng(83)
    sample_g = [5, 50]
    traces = np.sort(rng.choice(geo.ntr, 24, replace=False))
    slices = [3, 40]
    shape_m = (geo.ntau, geo.nq, geo.ntheta)
    ms = {i: rng.standard_normal(shape_m) for i in sample_g}
    _, dl = syn.shared_batch(gathers=sample_g)
    ds = dict(zip(sample_g, dl))
    d_ref = {i: ops.forward_traces(op, ms[i], traces) for i in sample_g}
    m_ref = {i: ops.adjoint_slices(op, ds[i], slices) for i in sample_g}
    tr_idx = torch.from_numpy(traces).cuda()
    sl_idx = torch.tensor(slices).cuda()
    errs = {}
    for prec in ("split_bf16", "fp32"):
        gp = gpu_plan(geo, ngather=G, precision=prec)
        tc = prec == "split_bf16"
        m_in = torch.zeros(shape_m + (G,) if tc else (G,) + shape_m, device="cuda")
        d_in = torch.zeros((geo.nt, geo.ntr, G) if tc else (G, geo.nt, geo.ntr), device="cuda")
        for i in sample_g:
            mt = torch.from_numpy(ms[i].astype(np.float32)).cuda()
            dt_ = torch.from_numpy(ds[i].astype(np.float32)).cuda()
            if tc:
                m_in[..., i] = mt
                d_in[..., i] = dt_
            else:
                m_in[i] = mt
                d_in[i] = dt_
        dg = gp.forward(m_in.reshape(-1))
        mg = gp.adjoint(d_in.reshape(-1))
        gp.status()
        for i in sample_g:
            if tc:
                dgi = dg.reshape(geo.nt, geo.ntr, G)[:, :, i]
                mgi = mg.reshape(shape_m + (G,))[..., i]
            else:
                dgi = dg.reshape(G, geo.nt, geo.ntr)[i]
                mgi = mg.reshape((G,) + shape_m)[i]
            ef = rel(host(dgi.index_select(1, tr_idx)), d_ref[i])
            ea = rel(host(mgi.index_select(2, sl_idx)), m_ref[i])
            errs[(prec, i)] = (ef, ea)
            assert ef < TOL_OP and ea < TOL_OP
        del dg, mg, m_in, d_in
        gp.close()
        del gp
        torch.cuda.empty_cache()
    print("relative L2 vs FP64 oracle (forward, adjoint):", errs)


def test_bounded_wait_reports_timeout_and_recovers():
    """Failure path of the tensor-core kernels without a GPU fault: under the
    test hook no matrix operation is issued, so every bounded wait runs out
    (20 ms of device time); the kernels flag it, release their tensor memory
    and return, aahrt_plan_status reports AAHRT_ERR_TIMEOUT, and the plan
    computes the same result as before once the hook is off."""
    from paper_2505_00387_gb300 import _lib as L
    g = syn.small_cube()
    G = 3
    gp = gpu_plan(g, ngather=G, precision="split_bf16")
    rng = np.random.default_rng(140)
    m = dev(interleave([rng.standard_normal(g.m.shape) for _ in range(G)]))
    d0 = gp.forward(m).clone()
    gp.status()
    L.aahrt_plan_test_stall(gp.handle, True)
    try:
        gp.forward(m)
        with pytest.raises(L.AahrtError) as err:
            gp.status()
        assert err.value.status == L.AAHRT_ERR_TIMEOUT
        gp.status()                              # the flag was cleared
    finally:
        L.aahrt_plan_test_stall(gp.handle, False)
    d1 = gp.forward(m)
    gp.status()
    assert torch.equal(d0, d1)
    fp = gpu_plan(g)                             # FP32 plans have no such wait
    with pytest.raises(L.AahrtError):
        L.aahrt_plan_test_stall(fp.handle, True)
