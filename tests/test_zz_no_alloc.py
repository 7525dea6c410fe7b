"""aahrt_forward_noalloc: the forward transform for callers that must not
allocate device memory during the call (code whose device heap belongs to an
external memory manager, or loops that forbid allocation on their hot path).
Its scratch lives in one fixed device array that plan creation loads and
looks up; its results must match aahrt_forward's on every kind of plan (the
FP32 spreading slice step, a deconvolutive plan, the direct-sum slice step,
the split-BF16 tensor-core contraction of several gathers).  Collected last
so that a run stopping at the first failure has already run every other
test; it also runs alone."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL_OP = 1e-4   # relative L2 tolerance of one operator application

KINDS = ["spread", "wavelet", "direct", "split_bf16"]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _plan(kind):
    from paper_2505_00387_gb300 import build
    build.build()
    from paper_2505_00387_gb300 import synthetic as syn
    from paper_2505_00387_gb300.plan import AahrtPlan
    g = syn.small_cube()
    if kind == "direct":
        gp = AahrtPlan(**g.geom_kwargs(), slice_interp="direct")
    elif kind == "split_bf16":
        gp = AahrtPlan(**g.geom_kwargs(), ngather=4, precision="split_bf16")
    else:
        gp = AahrtPlan(**g.geom_kwargs())
    if kind == "wavelet":
        t = (np.arange(31) - 15) * g.dt
        gp.set_wavelet(syn.ricker(t, 25.0).astype(np.float32), 15)
    return gp


@pytest.mark.parametrize("kind", KINDS)
def test_noalloc_forward_matches_forward_twice(kind):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_00387_gb300 import _lib as L
    gp = _plan(kind)
    rng = np.random.default_rng(90)
    stream = int(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        m = torch.from_numpy(rng.standard_normal(gp.model_len).astype(np.float32)).cuda()
        d_ref = torch.empty(gp.data_len, device="cuda")
        d_new = torch.full((gp.data_len,), float("nan"), device="cuda")
        L.aahrt_forward(gp.handle, m.data_ptr(), d_ref.data_ptr(), stream)
        L.aahrt_forward_noalloc(gp.handle, m.data_ptr(), d_new.data_ptr(), stream)
        torch.cuda.synchronize()
        a, b = d_new.cpu().numpy(), d_ref.cpu().numpy()
        assert np.all(np.isfinite(a)), f"{kind} call {call}: non-finite output"
        assert _rel(a, b) <= TOL_OP, f"{kind} call {call}: rel {_rel(a, b):.3e}"
    if kind == "split_bf16":
        gp.status()       # raises if a tensor-core wait ran out
    gp.close()


def test_noalloc_rejects_plans_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_00387_gb300 import _lib as L
    from paper_2505_00387_gb300 import synthetic as syn
    from paper_2505_00387_gb300.plan import AahrtPlan
    g = syn.paper_gather()
    gp = AahrtPlan(**g.geom_kwargs())
    need = 8 * (gp.info.xspec_len + gp.info.yspec_len) + 256
    assert need > L.AAHRT_NOALLOC_SCRATCH_BYTES
    m = torch.zeros(gp.model_len, device="cuda")
    d = torch.zeros(gp.data_len, device="cuda")
    with pytest.raises(L.AahrtError) as e:
        L.aahrt_forward_noalloc(gp.handle, m.data_ptr(), d.data_ptr())
    assert e.value.status == L.AAHRT_ERR_UNSUPPORTED
    assert "scratch" in str(e.value)
