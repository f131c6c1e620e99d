"""The allocation-free field sums (lbm_field_sums_static) against lbm_reduce.

lbm_field_sums_static exists for callers that cannot allocate device memory
at the point where they check mass and momentum (fixed memory pools, loops that
must not synchronise the device through cudaMalloc, hosts that own all GPU
memory): its partial sums live in a fixed array inside the library.  This
test feeds it caller-owned device arrays and compares two calls in a row with
the context's own reduction, through the C ABI.  The file name sorts last so
that a run stopping at the first failure has run every other test already.
"""
import numpy as np
import pytest

from paper_1711_03254_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_field_sums_static_matches_reduce():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_03254_gb300 import build
    build.build()
    from paper_1711_03254_gb300 import lbm

    n = 20
    batch = 3
    ts, r1s, r2s, us, ps = [], [], [], [], []
    for k in range(batch):
        t, r1, r2, u = W.droplet(n, n, n, 4.0 + k)
        t[:, 0, :] = W.SOLID
        r1[t == W.SOLID] = 0
        r2[t == W.SOLID] = 0
        ts.append(t), r1s.append(r1), r2s.append(r2), us.append(u)
        ps.append(dict(tau=(0.8 + 0.1 * k, 1.1), G=-1.8, rho_s=0.1 * k, g=(1e-5 * (k + 1), 0, 0)))
    t = np.stack(ts)
    sim = lbm.Sim(n, n, n, ps, precision="fp64")
    sim.set_geometry(t)
    sim.set_fields(np.stack(r1s), np.stack(r2s), np.stack(us))
    sim.step(25)
    a, b, v = sim.get_fields()
    ref = sim.reduce()  # [batch, 7]: M1 M2 Px Py Pz residual max|u|

    dev = torch.device("cuda:0")
    da = torch.from_numpy(a).to(dev)
    db = torch.from_numpy(b).to(dev)
    dv = torch.from_numpy(v).to(dev)
    dt = torch.from_numpy(t).to(dev)
    for _ in range(2):  # two calls in a row share the library's scratch array
        out = torch.full((batch, 6), float("nan"), dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream().cuda_stream
        lbm.lbm_field_sums_static(da.data_ptr(), db.data_ptr(), dv.data_ptr(), dt.data_ptr(), n * n * n, batch,
                                  out.data_ptr(), stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.allclose(got[:, :2], ref[:, :2], rtol=1e-12, atol=0)
        assert np.allclose(got[:, 2:5], ref[:, 2:5], rtol=1e-10, atol=1e-15)
        assert np.allclose(got[:, 5], ref[:, 6], rtol=1e-12, atol=0)


def test_field_sums_static_rejects_large_batch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_03254_gb300 import lbm
    dev = torch.device("cuda:0")
    x = torch.zeros(65 * 8, dtype=torch.float64, device=dev)
    t = torch.zeros(65 * 8, dtype=torch.uint8, device=dev)
    out = torch.zeros(65 * 6, dtype=torch.float64, device=dev)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_field_sums_static(x.data_ptr(), x.data_ptr(), x.data_ptr(), t.data_ptr(), 8, 65, out.data_ptr())
    assert e.value.status == 1
