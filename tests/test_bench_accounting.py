"""CPU tests of bench.py's accounting: the algorithmic bytes per stage (the
staged count every `roofline` and `pair_hbm` figure divides by) and the
tensor-core flops the split-BF16 contraction issues, against hand counts."""
import os
import sys
from types import SimpleNamespace

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def paper_gather_info():
    """Buffer lengths of the paper-scale gather's plan: nt = ntau = 1001,
    100 q x 36 azimuths, 2000 traces, 2048 bins."""
    return SimpleNamespace(model_len=1001 * 100 * 36, data_len=1001 * 2000,
                           xspec_len=2048 * 100 * 36, yspec_len=2048 * 2000)


def test_stage_bytes_paper_gather():
    sb = bench.stage_bytes(paper_gather_info())
    m, d = 4 * 1001 * 3600, 4 * 1001 * 2000
    x, y = 8 * 2048 * 3600, 8 * 2048 * 2000
    assert sb == [m + x, x + y, y + 2 * d, d + y, y + x, x + 4 * m, 0]
    assert sum(sb) == 463_097_600                # 463.1 MB per staged iteration
    assert sb[4] == 91_750_400                   # the slice adjoint's 91.8 MB


def test_launch_bytes_of_the_fused_iteration():
    info = paper_gather_info()
    sb = bench.stage_bytes(info)
    # fused solve of 100 iterations: no stage-3 launches, 100 data-side fused
    # launches, 100 model-side syntheses of which 99 also analyse the new z
    launches = [1, 100, 100, 0, 100, 100, 0]
    lb = bench.launch_bytes(info, launches, 100)
    m, d = 4 * info.model_len, 4 * info.data_len
    x, y = 8 * info.xspec_len, 8 * info.yspec_len
    assert lb[2] == 2 * y + d
    assert lb[5] == int(x + 4 * m + x * 99 / 100)
    assert lb[1] == sb[1] and lb[4] == sb[4]
    # unfused launches keep the staged count
    assert bench.launch_bytes(info, [100, 100, 100, 100, 100, 100, 0], 100) == sb


def test_tc_flops_hand_count():
    # 3 azimuth slices holding 130, 0 and 40 traces (all on the slice centres)
    ntheta = 3
    th = np.concatenate([np.full(130, 0.5), np.full(40, 2.5)]) * np.pi / ntheta
    hx, hy = 1000.0 * np.cos(th), 1000.0 * np.sin(th)
    nq, nbins, G = 40, 7, 8
    fwd, adj = bench.tc_flops(hx, hy, nq, ntheta, nbins, G)
    k = 3 * 2 * 16                               # three products, 2 flops, K = 16 per MMA
    gp = 8
    row_tiles = 2 + 0 + 1                        # ceil(130/128) + 0 + ceil(40/128)
    kchunks = 2                                  # ceil(40/32)
    assert fwd == nbins * row_tiles * kchunks * 4 * k * 128 * 4 * gp
    # adjoint chunks of 32 traces over slices (j, j-1): (130+40), (0+130), (40+0)
    chunks = 6 + 5 + 2
    assert adj == nbins * chunks * 1 * 4 * k * 128 * 2 * gp
    with pytest.raises(Exception):
        bench.tc_flops(hx, hy[:-1], nq, ntheta, nbins, G)


def test_gpu_dot_rel_helper_on_cpu_matrices():
    """The dot-test helper behind the shared-geometry arms' dot_test_rel: an
    exact transpose pair gives rounding-level values, a pair whose adjoint is
    off by one entry does not (run here on CPU tensors)."""
    import torch
    rng = np.random.default_rng(7)
    A = torch.from_numpy(rng.standard_normal((300, 200)).astype(np.float32))
    m = torch.from_numpy(rng.standard_normal(200).astype(np.float32))
    exact = bench.gpu_dot_rel(lambda x: A @ x, lambda y: A.T @ y, m, 3)
    assert exact < 1e-6
    B = A.clone()
    B[10, 20] += 1.0
    off = bench.gpu_dot_rel(lambda x: A @ x, lambda y: B.T @ y, m, 3)
    assert off > 1e-4


def test_traffic_record_follows_the_source_hash(tmp_path, monkeypatch):
    """A committed ncu record is reported only while the files that define
    its kernel hash to the recorded value: editing one of them hides it."""
    import hashlib
    import json
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k() {}\n")
    (tmp_path / "profiles").mkdir()
    rec = {"kernel": "k", "dram_bytes": 123, "files": ["k.cu"],
           "sha256": hashlib.sha256(src.read_bytes()).hexdigest()}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"kernels": {"st": rec}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_record("st")["dram_bytes"] == 123
    assert bench.traffic_record("other") is None
    src.write_text("__global__ void k() { }\n")
    assert bench.traffic_record("st") is None

