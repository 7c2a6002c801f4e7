"""Continuous-batching server: requests of mixed sizes, methods and storage
types submitted back to back overlap on the device, and every result equals
the standalone reconstruction of the same capture (with the same autotuned
launch shapes) bit for bit (same alone and in the mix). The memory budget covers resident plans and running workspaces."""
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
        plan.autotune()          # the server's launch shapes (the autotune cache is process-wide)
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
    plan.autotune()              # the launch shapes the server's plan will take from the shared cache
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


def test_plan_memory_counts_and_idle_plans_give_way():
    """The budget covers resident plans (radial kernels and tensor-core operand
    stores of phasor-field plans are tens of MB) as well as workspaces: with a
    budget that holds about two plans and a workspace, a mix over four plans
    evicts idle plans (least recently used first), never holds more than the
    budget, and every result still equals its standalone reconstruction."""
    from paper_2608_28183_gb300 import nlos
    shapes = []
    for k, nt in enumerate((256, 512, 384, 448)):
        g = synth.Geometry(32, 32, nt, 16e-12, 1.0, 1.0)
        kw = dict(n_depths=48, depth_min_m=0.4, depth_max_m=nt * g.bin_depth_m)
        shapes.append((g, kw))
    plans = [nlos.plan_for_capture(g, "pf", "f32", **kw) for g, kw in shapes]
    for p in plans:
        p.autotune()             # the launch shapes the server's plans will take from the shared cache
    # what a plan holds besides its own default workspace (the server's plans have none)
    sizes = [p.resident_bytes - p.workspace_bytes for p in plans]
    assert min(sizes) > 1 << 20                       # tables and kernels, not just the workspace
    budget = 2 * max(sizes) + 2 * max(p.workspace_bytes for p in plans) + (1 << 20)
    server = nlos.Server(memory_budget_bytes=budget, n_slots=2)
    rng = np.random.default_rng(7)
    order = [0, 1, 2, 3, 0, 2, 1, 3, 3, 0]
    outs, refs, tickets = [], [], []
    for i in order:
        g, kw = shapes[i]
        cap = synth.point_capture(g, [(rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2), 0.6, 1.0)], peak=200.0)
        x = to_device(cap.counts, torch.float32)
        refs.append(plans[i].reconstruct(x).clone())
        o = torch.full(plans[i].out_shape, float("nan"), device="cuda")
        outs.append(o)
        tickets.append(server.submit(nlos.desc_for_capture(g, "pf", "f32", **kw), x, o))
        m = server.memory()
        assert m["plan_bytes"] + m["workspace_bytes"] <= budget
    for t in tickets:
        server.wait(t)
    for o, r in zip(outs, refs):
        assert torch.equal(o, r)
    m = server.memory()
    assert m["evictions"] >= 2 and m["plan_bytes"] <= budget
    server.close()
