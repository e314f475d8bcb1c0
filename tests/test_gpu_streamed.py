"""GPU tests of StreamedBuilder: full builds of host-resident sets with the transfers overlapped
with the builds must equal build_octree on device copies of the same sets, bit for bit, for every
set of the sequence (the two slots alternate, so sets k and k+2 share buffers)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _sets(n, count):
    from paper_2307_06345_gb300 import workloads as w
    out = []
    for k in range(count):
        x, y, z = (w.clumps(n, 500 + k, n_clumps=20) if k % 2 else w.plummer(n, 600 + k))
        m = w.lognormal_masses(n, 700 + k)
        out.append(tuple(torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (x, y, z, m)))
    return out


@pytest.mark.parametrize("curve", [0, 1])
def test_streamed_equals_build_octree(lib, curve):
    n = 150_001
    sets = _sets(n, 5)
    sb = lib.StreamedBuilder(n, "cuda", curve=curve, ncrit=32)
    got = {}

    def keep(k, r):  # copy: the pinned result buffers are reused two sets later
        got[k] = {name: (v.clone() if torch.is_tensor(v) else v) for name, v in r.items()}

    h2d, d2h = sb.run(sets, on_result=keep)
    assert sorted(got) == list(range(len(sets)))
    assert h2d == len(sets) * n * 28
    for k, (x, y, z, m) in enumerate(sets):
        ref = lib.build_octree(x.cuda(), y.cuda(), z.cuda(), curve=curve, ncrit=32, masses=m.cuda())
        torch.cuda.synchronize()
        r = got[k]
        assert r["n_leaves"] == ref["n_leaves"]
        for name in sb.OUT:
            assert torch.equal(r[name], ref[name].reshape(-1).cpu()), (k, name)
    assert d2h == sum(sum(got[k][name].numel() * got[k][name].element_size() for name in sb.OUT) for k in got)


def test_streamed_rejects_wrong_sets(lib):
    sb = lib.StreamedBuilder(1000, "cuda")
    x = torch.zeros(999, dtype=torch.float64)
    with pytest.raises(ValueError):
        sb.run([(x, x, x, torch.zeros(999, dtype=torch.float32))])
    with pytest.raises(ValueError):
        sb.run([(torch.zeros(1000, dtype=torch.float64, device="cuda"),) * 3 + (torch.zeros(1000),)])


@pytest.mark.parametrize("count", [1, 2])
def test_streamed_short_sequences(lib, count):
    n = 10_000
    sets = _sets(n, count)
    sb = lib.StreamedBuilder(n, "cuda", curve=1, ncrit=16)
    got = {}
    sb.run(sets, on_result=lambda k, r: got.setdefault(k, r["NK"].clone()))
    assert sorted(got) == list(range(count))
    for k, (x, y, z, m) in enumerate(sets):
        ref = lib.build_octree(x.cuda(), y.cuda(), z.cuda(), curve=1, ncrit=16, masses=m.cuda())
        assert torch.equal(got[k], ref["NK"].cpu())
