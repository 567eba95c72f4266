"""The allocation-free spreading entry point (mb_spread_static) against mb_spread.

mb_spread_static serves callers that cannot allocate device memory: it keeps its binning
scratch in a fixed array compiled into the library.  This file is collected last on purpose,
so that a run stopping at the first failure has already run every other test; it also passes
when run alone in a fresh process (the scratch address is set up on the first call).
"""
import numpy as np
import pytest

from helpers import TOL, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_1407_5600_gb300 as mb  # noqa: E402
from paper_1407_5600_gb300 import workloads as wl  # noqa: E402


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape,h,n", [((16, 32, 64), 1.0, 20011), ((8, 8, 8), 0.5, 300)])
def test_static_spread_matches_spread_on_two_calls_in_a_row(prec, shape, h, n):
    nz, ny, nx = shape
    d = mb.GridDesc(nx, ny, nz, h=h, precision=prec)
    dt = torch.float64 if prec == 1 else torch.float32
    stream = torch.cuda.current_stream()
    ctx = mb.create_grid(d, stream)
    try:
        for call, seed in enumerate((n, n + 7)):
            q, F, _ = wl.random_blobs(n, shape, seed=seed, h=h)
            q[0] = [-0.25 * h, 1e3 * h, nx * h]           # outside the box: wrapped
            qd = torch.as_tensor(q, device="cuda")
            Fd = torch.as_tensor(F, device="cuda")
            ref = torch.empty((1, 3) + shape, dtype=dt, device="cuda")
            out = torch.full((1, 3) + shape, float("nan"), dtype=dt, device="cuda")
            mb.spread(ctx, qd, Fd, ref)
            mb.spread_static(d, qd, Fd, out, stream)
            torch.cuda.synchronize()
            err = rel_l2(out.cpu().numpy(), ref.cpu().numpy())
            assert err < TOL[prec], (call, err)
    finally:
        mb.destroy(ctx)


def test_static_spread_rejects_sizes_beyond_its_scratch():
    d = mb.GridDesc(8, 8, 8)
    q = torch.zeros((262145, 3), dtype=torch.float64, device="cuda")
    out = torch.empty((1, 3, 8, 8, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(mb.MBError) as ei:
        mb.spread_static(d, q, q, out)
    assert ei.value.status == 1 and "262144" in str(ei.value)
    with pytest.raises(mb.MBError) as ei:
        mb.spread_static(d, np.zeros((4, 3)), np.zeros((4, 3)), out)
    assert ei.value.status == 1 and "device pointers" in str(ei.value)
