"""The algorithmic-byte model behind the benchmark's rooflines (CPU only).

Per launch a stage moves its unique input plus its unique output in the
stored element sizes. With V = a b n voxels and V' = (a + 1) b n (kx in
[0, a] after the real-input x transform), float32 storage:
  fused x-forward then y-forward        4V + 16V'
  Stolt stage (inverse temporal last)   16V' + 32V
  fused y-inverse then x-inverse        32V + 8V (complex kept spectrum)
  inverse temporal transform last       8V + 4V
and the method's own model (Sec. 4.2: input, half spectrum written and read,
post-Stolt spectrum written and read, output) is 104V, 54V with 16-bit
storage.
"""
import importlib.util
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_model_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("a,b,n", [(256, 256, 512), (32, 32, 256), (64, 128, 1024)])
def test_stage_bytes_follow_the_per_stage_formulas(bench, a, b, n):
    V = a * b * n
    Vp = (a + 1) * b * n
    sb = bench.stage_bytes(a, b, n, "f32", zlast=True)
    assert sb["fk_xy_forward"] == 4 * V + 16 * Vp
    assert sb["fk_stolt"] == 16 * Vp + 32 * V
    assert sb["fk_yx_inverse"] == 32 * V + 8 * V
    assert sb["fk_z_inverse"] == 8 * V + 4 * V
    # the fused inverse writes |psi|^2 where the temporal inverse is not last
    assert bench.stage_bytes(a, b, n, "f32", zlast=False)["fk_yx_inverse"] == 32 * V + 4 * V
    # the separate passes
    assert sb["fk_x_forward"] == 4 * V + 8 * Vp
    assert sb["fk_y_forward"] == 8 * Vp + 16 * Vp
    assert sb["fk_y_inverse"] == 32 * V + 16 * V
    assert sb["fk_x_inverse"] == 16 * V + 4 * V


def test_totals_against_the_method_model(bench):
    a, b, n = 256, 256, 512
    V = a * b * n
    sb = bench.stage_bytes(a, b, n, "f32", zlast=True)
    four = sb["fk_xy_forward"] + sb["fk_stolt"] + sb["fk_yx_inverse"] + sb["fk_z_inverse"]
    separate = sb["fk_x_forward"] + sb["fk_y_forward"] + sb["fk_stolt_z"] + sb["fk_y_inverse"] + sb["fk_x_inverse"]
    assert bench.pipeline_bytes(a, b, n, "f32") == 104 * V
    assert bench.pipeline_bytes(a, b, n, "f16") == 54 * V
    # the four-stage form moves the 8V kept spectrum twice more than the model
    assert four / V == pytest.approx(120 + 32 / a)
    assert separate / V == pytest.approx(152 + 48 / a)
    # 16-bit storage halves every complex and real element
    s16 = bench.stage_bytes(a, b, n, "f16", zlast=True)
    for k in ("fk_xy_forward", "fk_stolt", "fk_yx_inverse"):
        assert s16[k] * 2 == sb[k]


def test_committed_traffic_summary_uses_the_same_algorithmic_bytes(bench):
    with open(os.path.join(ROOT, "profiles", "fk_256x256x512_traffic.json")) as f:
        d = json.load(f)
    sb = bench.stage_bytes(256, 256, 512, "f32", zlast=True)
    # each stage's figure is tied to the sources its kernel is built from
    assert set(d["kernel_hashes"]) == set(bench.STAGE_SOURCES) == set(d["per_stage"])
    for stage, rec in d["per_stage"].items():
        assert rec["algorithmic_bytes"] == sb[stage], stage
        assert d["dram_bytes_per_launch"][stage] == rec["dram_read"] + rec["dram_write"]
        assert rec["traffic_over_algorithmic"] == pytest.approx(
            (rec["dram_read"] + rec["dram_write"]) / rec["algorithmic_bytes"], abs=1e-3)


def test_traffic_is_reported_only_while_the_stage_sources_match(bench, tmp_path):
    d = {"kernel_hashes": {s: bench.stage_hash(s) for s in bench.STAGE_SOURCES},
         "dram_bytes_per_launch": {s: 1000 + i for i, s in enumerate(bench.STAGE_SOURCES)}}
    d["kernel_hashes"]["fk_stolt"] = "0" * 16          # as if the Stolt kernel changed since
    path = tmp_path / "traffic.json"
    path.write_text(json.dumps(d))
    assert bench.profiled_traffic("fk_yx_inverse", str(path)) == d["dram_bytes_per_launch"]["fk_yx_inverse"]
    assert bench.profiled_traffic("fk_stolt", str(path)) is None
    assert bench.profiled_traffic("no_such_stage", str(path)) is None
    assert bench.profiled_traffic("fk_yx_inverse", str(tmp_path / "missing.json")) is None
