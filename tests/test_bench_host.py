"""Host logic of bench.py that needs no GPU: the DRAM-traffic figure of the
roofline is taken from the committed ncu summary only while the fused
kernel's code is the code that was profiled (comments may change)."""
import json
import os

import bench


def _tree(tmp_path, k_tc, ptx):
    csrc = tmp_path / "paper_1412_4907_gb300" / "csrc"
    csrc.mkdir(parents=True)
    files = dict.fromkeys(bench.KERNEL_SOURCES, "#pragma once\n")
    files[bench.KERNEL_SOURCES[0]] = k_tc
    files["ptx.cuh"] = ptx
    for name, text in files.items():
        (csrc / name).write_text(text)
    return str(tmp_path)


def test_source_hash_ignores_comments_not_code(tmp_path, monkeypatch):
    code = "int f(int x)\n{\n    return x + 1;   // one\n}\n/* block\n comment */\n"
    monkeypatch.setattr(bench, "ROOT", _tree(tmp_path / "a", code, "#pragma once\n"))
    h0 = bench.kernel_source_sha()
    monkeypatch.setattr(bench, "ROOT", _tree(tmp_path / "b", code.replace("// one", "// changed note")
                                             .replace("block\n comment", "other"), "#pragma once\n"))
    assert bench.kernel_source_sha() == h0
    monkeypatch.setattr(bench, "ROOT", _tree(tmp_path / "c", code.replace("x + 1", "x + 2"), "#pragma once\n"))
    assert bench.kernel_source_sha() != h0


def test_profiled_traffic_needs_matching_source(tmp_path, monkeypatch):
    root = _tree(tmp_path, "int g;\n", "#pragma once\n")
    monkeypatch.setattr(bench, "ROOT", root)
    prof = tmp_path / "k_tc_config2.json"
    monkeypatch.setattr(bench, "PROFILE", str(prof))
    assert bench.profiled_traffic() is None                     # no capture
    prof.write_text(json.dumps({"dram_bytes_per_launch": 123.0, "source_sha": bench.kernel_source_sha()}))
    assert bench.profiled_traffic() == 123.0
    prof.write_text(json.dumps({"dram_bytes_per_launch": 123.0, "source_sha": "0" * 16}))
    assert bench.profiled_traffic() is None                     # taken on other code
    assert os.path.exists(str(prof))
