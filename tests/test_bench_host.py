"""Host logic of bench.py (CPU only): the default line's config object, the
algorithmic byte and flop models, and the source-hash gate on the committed
ncu traffic figure."""
import argparse
import hashlib
import os

import bench
from synthetic import workload


def _args(**kw):
    base = dict(basis="sdme_h", precision="mixed")
    base.update(kw)
    return argparse.Namespace(**base)


def test_config_names_the_cantilever_and_its_sizes():
    w = workload("beam_p8")
    cfg = bench.workload_config(_args(), w, 1)
    assert "6502275 DOFs" in cfg["workload"] and "64x8x8 hexes, P=8" in cfg["workload"]
    assert cfg["parallelism"] == "single" and cfg["global_batch"] == 1
    # float32 state: 10 words x 10^3 points x 4,096 elements x 4 bytes
    assert "156 MB" in cfg["l2"]
    assert "312 MB" in bench.workload_config(_args(precision="fp64"), w, 1)["l2"]
    assert bench.workload_config(_args(), w, 2)["parallelism"] == "replicas"


def test_tangent_bytes_match_the_layout():
    # state (10 words per Gauss point) + x read + y read and written
    P, nelem, ndof = 8, 4096, 6502275
    assert bench.tangent_bytes(P, nelem, ndof, 4, 4) == 10 * 1000 * nelem * 4 + 3 * ndof * 4
    assert bench.tangent_bytes(P, nelem, ndof, 4, 4) == 241867300


def test_traffic_is_reported_only_for_the_captured_sources(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2104_13466_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for i, f in enumerate(bench.KERNEL_SOURCES):
        (csrc / f).write_bytes(b"source %d\n" % i)
    h = hashlib.sha256()
    for f in bench.KERNEL_SOURCES:
        h.update((csrc / f).read_bytes())
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "tangent_kernel_f32_beam_p8.md").write_text(
        "summary\n\n    traffic_bytes_per_launch: 123456\n    kernel_source_sha256: %s\n" % h.hexdigest())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("mixed") == 123456.0
    assert bench.profiled_traffic("fp64") is None          # no float64 summary in this tree
    (csrc / bench.KERNEL_SOURCES[0]).write_bytes(b"changed\n")
    assert bench.profiled_traffic("mixed") is None         # sources changed since the capture


def test_committed_summaries_carry_the_gate_fields():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for name in ("tangent_kernel_f32_beam_p8.md", "tangent_kernel_f64_beam_p8.md"):
        text = open(os.path.join(root, "profiles", name)).read()
        assert "traffic_bytes_per_launch:" in text and "kernel_source_sha256:" in text
        assert "ncu " in text and "--clock-control none" in text


def test_flop_model_figures():
    # the even-odd count quoted with the roofline: 588,852 flops per P = 8
    # element, 2.41 GFLOP per launch on the 4,096-element cantilever; the
    # plain contraction count is 1.46x that
    assert bench.tangent_flops_per_element(8) == 588852
    assert bench.tangent_flops_per_element(8) * 4096 == 2411937792
    n, Q = 9, 10
    plain = 4 * 3 * (n ** 3 * Q + n ** 2 * Q ** 2 + n * Q ** 3 + 3 * Q ** 4) + 207 * Q ** 3
    assert abs(plain / bench.tangent_flops_per_element(8) - 1.46) < 0.01
    # the nodal basis pays the pairing adds on the mode-side lines
    assert bench.tangent_flops_per_element(8, nodal=True) > bench.tangent_flops_per_element(8)
    # the roofline's unit is the plain count: 859,680 flops per P = 8 element
    assert bench.algorithmic_flops_per_element(8) == plain == 859680
    assert bench.algorithmic_flops_per_element(8) * 4096 == 3521249280
