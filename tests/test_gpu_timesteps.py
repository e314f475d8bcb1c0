"""GPU parity of the time-step driver: several runs moved by small Gaussian displacements, every
step rebuilt from the previous step's leaves (warm start, Sec. 4) in a box fixed at step 0.

Every warm rebuild equals a cold rebuild of the same step (the balanced tree is unique), and
sampled runs and steps equal the oracle's build from the raw coordinates."""
import numpy as np
import pytest
import torch

from _gpu_util import dev, i32, u32, u64

pytestmark = pytest.mark.gpu


def _equal(a, b, keys):
    for k in keys:
        assert torch.equal(a[k], b[k]), k


def test_time_steps_warm_equals_cold_and_oracle(lib, oracle):
    from paper_2307_06345_gb300 import workloads as w
    runs, n, steps = 8, 1 << 18, 6
    parts = [w.plummer(n, w.BASE_SEED + 4 + r) for r in range(runs)]
    x = np.concatenate([p[0] for p in parts])
    y = np.concatenate([p[1] for p in parts])
    z = np.concatenate([p[2] for p in parts])
    off = (np.arange(runs + 1) * n).astype(np.int64)
    X, Y, Z, OFF = dev(x), dev(y), dev(z), dev(off)
    st = lib.TimeStepper(X, Y, Z, OFF, curve=lib.HILBERT, ncrit=64)
    boxes = st.boxes.cpu().numpy()
    side0 = float(boxes[0, 3]) / 1.2
    for step in range(steps):
        if step > 0:
            dx, dy, dz = w.displacement(x.size, w.BASE_SEED + 100 + step, 1e-3 * side0)
            x, y, z = x + dx, y + dy, z + dz
            X.copy_(dev(x)), Y.copy_(dev(y)), Z.copy_(dev(z))
        warm = st.rebuild(warm=step > 0)
        cold = lib.build_octrees_batched(X, Y, Z, OFF, curve=lib.HILBERT, ncrit=64, boxes=st.boxes)
        torch.cuda.synchronize()
        _equal(warm, cold, ["elements", "element_offsets", "leaf_counts", "NK", "CO", "LO", "node_counts"])
        if step > 0:
            assert warm["iters"] <= 4  # a slowly moving distribution needs few passes
        check = range(runs) if step in (0, steps - 1) else [0]
        eo, no = warm["element_offsets_host"], warm["node_offsets_host"]
        E, NK, counts = u64(warm["elements"]), u64(warm["NK"]), u32(warm["node_counts"])
        for r in check:
            a, b = off[r], off[r + 1]
            lo = boxes[r, :3]
            inside = np.all((np.stack([x[a:b], y[a:b], z[a:b]]) >= lo[:, None]) &
                            (np.stack([x[a:b], y[a:b], z[a:b]]) < lo[:, None] + boxes[r, 3]))
            assert inside  # the padded box still holds every particle: nothing is clamped
            ref = oracle.full_build(x[a:b], y[a:b], z[a:b], oracle.HILBERT, 64, box=boxes[r])
            assert np.array_equal(E[eo[r]: eo[r + 1]], ref["K"])
            assert np.array_equal(NK[no[r]: no[r + 1]], ref["NK"])
            assert np.array_equal(counts[no[r]: no[r + 1]], ref["counts"])
