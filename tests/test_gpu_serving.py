"""Continuous-batching server: requests of mixed sizes, methods and storage
types submitted back to back overlap on the device, and every result equals
the standalone reconstruction of the same capture bit for bit (same alone and
in the mix). Admission is by workspace footprint under the memory budget."""
import numpy as np
import pytest

from paper_2608_28183_gb300 import synth
from tests.gpu_util import to_device

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def library():
    from paper_2608_28183_gb300 import build, nlos
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return nlos.load_library()


def _requests(n, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        side = int(rng.choice([16, 32, 64]))
        nt = int(rng.choice([256, 512]))
        method = "fk" if k % 2 == 0 else "pf"
        storage = "f16" if rng.random() < 0.5 else "f32"
        g = synth.Geometry(side, side, nt, 16e-12, 1.0, 1.0)
        kw = {} if method == "fk" else dict(n_depths=32, depth_min_m=0.4, depth_max_m=nt * g.bin_depth_m)
        pts = np.array([(rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), rng.uniform(0.4, 0.9) * nt * g.bin_depth_m, 1.0)])
        cap = synth.render(g, synth.Scene(points=pts), peak=300.0, background=0.5, seed=100 + k)
        out.append((g, method, storage, kw, cap))
    return out


def test_results_identical_alone_and_in_the_mix():
    from paper_2608_28183_gb300 import nlos
    reqs = _requests(16)
    server = nlos.Server(memory_budget_bytes=4 << 30, n_slots=4)
    inputs, outputs, tickets, alone = [], [], [], []
    for g, m, st, kw, cap in reqs:
        desc = nlos.desc_for_capture(g, m, st, **kw)
        server.preload(desc)
        plan = nlos.plan_for_capture(g, m, st, **kw)
        x = to_device(cap.counts, plan.input_dtype())
        alone.append(plan.reconstruct(x).clone())
        inputs.append((desc, x))
        outputs.append(torch.full(plan.out_shape, float("nan"), device="cuda"))
    torch.cuda.synchronize()
    for (desc, x), o in zip(inputs, outputs):
        tickets.append(server.submit(desc, x, o))
    lat = [server.wait(t) for t in tickets]
    for o, a in zip(outputs, alone):
        assert torch.equal(o, a)
    st = server.stats()
    assert st["completed"] == len(reqs) and st["p50_ms"] <= st["p99_ms"] and all(v > 0 for v in lat)
    server.close()


def test_budget_admission_serialises_and_rejects():
    from paper_2608_28183_gb300 import nlos
    g = synth.Geometry(64, 64, 512, 16e-12, 1.0, 1.0)
    plan = nlos.plan_for_capture(g, "fk", "f32")
    need = plan.workspace_bytes
    server = nlos.Server(memory_budget_bytes=need + need // 2, n_slots=4)   # one at a time fits
    desc = nlos.desc_for_capture(g, "fk", "f32")
    caps = [synth.point_capture(g, [(0.05 * k, 0.0, 0.6, 1.0)], peak=100.0) for k in range(4)]
    xs = [to_device(c.counts, torch.float32) for c in caps]
    outs = [plan.empty_volume() for _ in caps]
    ts = [server.submit(desc, x, o) for x, o in zip(xs, outs)]
    for t in ts:
        server.wait(t)
    for x, o in zip(xs, outs):
        assert torch.equal(o, plan.reconstruct(x))
    small = nlos.Server(memory_budget_bytes=need // 4, n_slots=2)
    with pytest.raises(nlos.NlosError) as e:
        small.submit(desc, xs[0], outs[0])
    assert e.value.status == 2
    server.close()
    small.close()
