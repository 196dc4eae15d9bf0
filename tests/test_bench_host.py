"""Host logic of bench.py (no GPU): the code-only hash that keys a committed
ncu capture to the kernel sources, the lookup of the captured DRAM traffic,
and the algorithmic-bytes formula of the roofline."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_code_only_drops_comments_and_layout_but_keeps_literals():
    src = ('int a = 1; // one\n/* block\n comment */ const char* s = "x // y /* z */";\n'
           "char c = '/';   char q = '\\'';  int  b=2;\n")
    out = bench._code_only(src)
    assert out == 'int a = 1; const char* s = "x // y /* z */"; char c = \'/\'; char q = \'\\\'\'; int b=2;'
    # a comment-only edit leaves the code text alone; a code edit does not
    assert bench._code_only(src.replace("// one", "// two, longer\n   ")) == out
    assert bench._code_only(src.replace("b=2", "b=3")) != out


def test_captured_traffic_follows_the_code_hash(tmp_path, monkeypatch):
    # the hash covers the code of the sampler kernels' sources and the ABI
    # header: comments do not count, and neither do the other kernels' files
    csrc = tmp_path / "paper_2305_14306_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "include").mkdir()
    (tmp_path / "profiles").mkdir()
    for f in bench.SAMPLER_SOURCES:
        (csrc / f).write_text(f"// {f}\nint x_{len(f)} = 1;\n")
    (tmp_path / "include" / "hav.h").write_text("int abi = 1;\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.source_hash()
    prof = tmp_path / "profiles" / "hav_chain_kernel_w.md"
    prof.write_text(f"x\n\nsource_hash: {h}\ndram_bytes_per_call: 12345\n")
    assert bench.profiled_traffic("w") == 12345
    assert bench.profiled_traffic("other") is None
    k = csrc / "hav_sampler.cu"
    k.write_text(k.read_text() + "/* reworded comment */\n")
    (csrc / "hav_group.cu").write_text("__global__ void g() {}\n")  # another kernel's file
    assert bench.source_hash() == h and bench.profiled_traffic("w") == 12345
    (csrc / "hav_device.cuh").write_text("#define X 1\n")  # a device header of the sampler
    assert bench.source_hash() != h and bench.profiled_traffic("w") is None
    (csrc / "hav_device.cuh").write_text("// hav_device.cuh\nint x_14 = 1;\n")
    assert bench.source_hash() == h
    (tmp_path / "include" / "hav.h").write_text("int abi = 2;\n")  # the ABI header
    assert bench.source_hash() != h


def test_algorithmic_bytes_by_hand():
    # two levels, two layers: n = 1000 -> m = 200 -> m = 50
    def tr(m_l, n_in, iters):
        return {"m_l": m_l, "n_in": n_in, "iters": iters}
    traces = [tr(40, 1000, 5), tr(160, 960, 7), tr(10, 200, 3), tr(0, 190, 0)]
    got = bench.algorithmic_bytes(traces, [1000, 200], [200, 50], 2)
    want = (6 * 12 * 1000 + 8 * (12 * 960 + 1000 // 8) + 4 * 200
            + 4 * 12 * 200 + 4 * 50)  # an empty layer reads nothing
    assert got == want


def test_whole_job_single_rank():
    t, v = bench.whole_job(0.5, 2_000_000, 1)
    assert t == 0.5 and abs(v - 4.0) < 1e-12


def test_clock_sampler_without_nvidia_smi_cleans_up(monkeypatch):
    def no_smi(*a, **k):
        raise FileNotFoundError("nvidia-smi")
    monkeypatch.setattr(bench.subprocess, "Popen", no_smi)
    c = bench.Clocks(0)
    name = c.f.name
    out = c.stop()
    assert out["samples"] == 0 and out["sm_mhz"] is None and not os.path.exists(name)
    assert not bench.clocks_bad(out)


def test_clocks_bad_rules():
    ok = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}
    assert not bench.clocks_bad(ok)
    assert not bench.clocks_bad({**ok, "reasons": ["sw_power_cap"]})  # kept and noted
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert bench.clocks_bad({**ok, "reasons": [r]})
    assert bench.clocks_bad({**ok, "sm_mhz": 1000.0})  # stuck well below max with no reason
