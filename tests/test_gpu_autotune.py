"""The tile autotuner of the batched SIMT products (rsvd_autotune_*): with tuning on,
the first call of each shape class times the candidate tiles and caches the fastest;
results are bit-identical with and without tuning (every tile sums each output over K in
the same order), and a cached choice is used inside a graph capture."""
import numpy as np
import pytest

from gpu_util import need_gpu, torch
from paper_1710_01463_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    need_gpu()
    from paper_1710_01463_gb300 import _lib, api
    return _lib, api


def test_tuned_tiles_give_identical_results(mods, tmp_path):
    _lib, api = mods
    lib = _lib.load()
    shapes, f = inputs.sector_shapes(N=6, lo=100, hi=700, seed=11)
    As = [torch.from_numpy(inputs.spectral_matrix(m, n, inputs.power_spectrum(min(m, n), 1.2, fb), 50 + b))
          .float().cuda() for b, ((m, n), fb) in enumerate(zip(shapes, f))]
    ks = [min(40, *A.shape) for A in As]
    lib.rsvd_autotune_clear()
    plan = api.BatchedPlan([A.shape for A in As], ks, 8, 2, 3, 0, torch.float32, "cuda", chi_global=100)
    plan.run(As)
    torch.cuda.synchronize()
    ref = [s.clone() for s in plan.S] + [u.clone() for u in plan.U]
    assert lib.rsvd_autotune_entries() == 0
    lib.rsvd_autotune_enable(1)
    try:
        plan.run(As)
        torch.cuda.synchronize()
    finally:
        lib.rsvd_autotune_enable(0)
    n = lib.rsvd_autotune_entries()
    assert n > 0
    for a, b in zip([s for s in plan.S] + [u for u in plan.U], ref):
        assert torch.equal(a, b)
    # cached choices inside a capture
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.run(As)
    for s in plan.S:
        s.zero_()
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(plan.S, ref):
        assert torch.equal(a, b)
    path = tmp_path / "tiles.txt"
    assert lib.rsvd_autotune_save(str(path).encode()) == 0
    lib.rsvd_autotune_clear()
    assert lib.rsvd_autotune_load(str(path).encode()) == n
    lib.rsvd_autotune_clear()


def test_wide_fp32_tile_bit_identical(mods, tmp_path):
    # the 128 x 128 FP32 tile (8 x 8 outputs per thread, 128-bit shared loads; tile choice 3)
    # forced for every FP32 product class of a batched FP32 RSVD with ragged shapes: the
    # same bits as the default tiles, because every tile sums each output over K in the
    # same order
    _lib, api = mods
    lib = _lib.load()
    shapes = [(300, 520), (700, 260), (130, 900), (1030, 1000), (257, 257)]
    As = [torch.from_numpy(inputs.spectral_matrix(m, n, inputs.power_spectrum(min(m, n), 1.0, 1.0), 70 + b))
          .float().cuda() for b, (m, n) in enumerate(shapes)]
    ks = [40, 40, 40, 120, 64]
    lib.rsvd_autotune_clear()
    plan = api.BatchedPlan([A.shape for A in As], ks, 8, 2, 7, 0, torch.float32, "cuda")
    plan.run(As)
    torch.cuda.synchronize()
    ref = [s.clone() for s in plan.S] + [u.clone() for u in plan.U] + [v.clone() for v in plan.Vt]
    lib.rsvd_autotune_enable(1)
    try:
        plan.run(As)
        torch.cuda.synchronize()
    finally:
        lib.rsvd_autotune_enable(0)
    path = tmp_path / "tiles.txt"
    assert lib.rsvd_autotune_save(str(path).encode()) == 0
    lines, forced = [], 0
    for line in path.read_text().splitlines():
        f = line.split()
        if not line.startswith("#") and f[0] == "4" and f[1] == "4":
            f[-1] = "3"
            forced += 1
        lines.append(" ".join(f))
    assert forced > 0
    path.write_text("\n".join(lines) + "\n")
    lib.rsvd_autotune_clear()
    try:
        assert lib.rsvd_autotune_load(str(path).encode()) == len([x for x in lines if not x.startswith("#")])
        for s in plan.S:
            s.zero_()
        plan.run(As)
        torch.cuda.synchronize()
        for a, b in zip([s for s in plan.S] + [u for u in plan.U] + [v for v in plan.Vt], ref):
            assert torch.equal(a, b)
    finally:
        lib.rsvd_autotune_clear()
