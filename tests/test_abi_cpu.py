"""The C-ABI library builds, loads and exports every symbol that include/*.h declares,
and rejects invalid arguments before touching the GPU (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(pgg_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1704_08098_gb300 import build, pgg
    build.build()
    return pgg.load()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("pgg_create", "pgg_seed", "pgg_step_mcs", "pgg_count_coop", "pgg_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_argument_validation_without_gpu(lib):
    from paper_1704_08098_gb300 import pgg
    h = ctypes.c_void_p()
    assert lib.pgg_create(ctypes.byref(h), 30, 4.0, 0.5, pgg.U8, None) == pgg.PGG_ERR_ARG
    assert "multiple of 4" in pgg.last_error()
    assert lib.pgg_create(ctypes.byref(h), 48, 4.0, 0.5, pgg.BITPACK, None) == pgg.PGG_ERR_ARG
    assert lib.pgg_create(ctypes.byref(h), 64, -1.0, 0.5, pgg.U8, None) == pgg.PGG_ERR_ARG
    assert lib.pgg_create(ctypes.byref(h), 64, 4.0, 0.0, pgg.U8, None) == pgg.PGG_ERR_ARG
    assert lib.pgg_create(ctypes.byref(h), 64, 4.0, 0.5, 7, None) == pgg.PGG_ERR_ARG
    assert lib.pgg_create(None, 64, 4.0, 0.5, pgg.U8, None) == pgg.PGG_ERR_ARG
    assert h.value is None
    assert lib.pgg_seed(None, 1, 0.5) == pgg.PGG_ERR_ARG
    assert lib.pgg_step_mcs(None, 1, None) == pgg.PGG_ERR_ARG
    assert lib.pgg_set_game(None, pgg.GAME_PAIRWISE, None) == pgg.PGG_ERR_ARG
    assert lib.pgg_get_game(None, None, None) == pgg.PGG_ERR_ARG
    assert lib.pgg_set_lattice_packed(None, None, 0) == pgg.PGG_ERR_ARG
    assert lib.pgg_get_lattice_packed(None, None, None) == pgg.PGG_ERR_ARG
    assert lib.pgg_stage_lattice_packed(None, None, 0) == pgg.PGG_ERR_ARG
    assert lib.pgg_set_kernel_timing(None, 1) == pgg.PGG_ERR_ARG
    assert lib.pgg_kernel_time(None, None, None) == pgg.PGG_ERR_ARG
    lib.pgg_destroy(None)
    assert lib.pgg_version().decode().startswith("pgg-gb300")


def test_product_path_never_imports_the_oracle():
    """The library and its binding must not reach the CPU oracle (no fallback)."""
    pkg = os.path.join(ROOT, "paper_1704_08098_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if path.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            text = open(path).read()
            assert "import oracle" not in text and "from oracle" not in text, path
            assert "pgg_oracle" not in text and "liboracle" not in text, path


def test_stored_counters_match_the_current_kernel_sources():
    """bench.py's roofline takes per-launch instruction and DRAM counts from a table keyed by a
    hash of the kernel's sources (stale counts must not be reported for a changed kernel): the
    table holds entries for the current resident and direct sources."""
    import bench
    for kernel in ("resident", "direct"):
        h = bench.kernel_source_hash(kernel)
        assert any(k.split(":")[1] == h and k.split(":")[0].startswith(kernel) for k in bench.NCU), kernel
    for key, v in bench.NCU.items():
        assert v["alu_warp_inst"] > 0 and v["dram_bytes"] > 0, key


def test_kernel_code_hash_ignores_comments_only(tmp_path):
    """The counter key hashes the kernel sources without their // comments; that is sound only if
    no "//" stands inside a string literal (an even number of quotes before every "//"), and it must
    change with the code."""
    import bench
    csrc = os.path.join(ROOT, "paper_1704_08098_gb300", "csrc")
    for name in ("pgg_kernels_resident.cu", "pgg_kernels_direct.cu", "pgg_unit.cuh", "pgg_device.cuh"):
        for line in open(os.path.join(csrc, name)):
            if "//" in line:
                assert line.split("//", 1)[0].count('"') % 2 == 0, (name, line)
    src = "int a = 1;  // one\n// only a comment\n\nint b = 2;\n"
    path = str(tmp_path / "probe.cu")
    open(path, "w").write(src)
    base = bench.kernel_code(path)
    open(path, "w").write(src.replace("// one", "// another") + "// more\n")
    assert bench.kernel_code(path) == base
    open(path, "w").write(src.replace("int b = 2;", "int b = 3;"))
    assert bench.kernel_code(path) != base


def test_binding_fails_loudly_without_the_library(monkeypatch):
    """No fallback: with the CUDA library absent the binding raises instead of computing anything."""
    from paper_1704_08098_gb300 import pgg
    monkeypatch.setattr(pgg, "_lib", None)
    monkeypatch.setattr(pgg, "LIB_PATH", os.path.join(os.path.dirname(pgg.LIB_PATH), "absent.so"))
    with pytest.raises(RuntimeError, match="CUDA library not built"):
        pgg.load()
    with pytest.raises(RuntimeError, match="CUDA library not built"):
        pgg.Lattice(64, 4.0, 0.5)


def test_host_threshold_tables_match_the_oracle(lib):
    """The library's host-built adoption tables (its own statement of Eq. (3) and the payoff rules,
    pgg_threshold_table, no device needed) equal the oracle's thresholds entry by entry, for the
    group game and the pairwise game of Section VI, including the K -> 0 and K -> infinity limits."""
    import oracle
    from paper_1704_08098_gb300 import pgg
    o = oracle.Oracle()
    for r, K in ((4.0, 0.5), (3.7443, 0.5), (3.98, 0.5), (5.0, 0.1), (4.2, 1e-6), (3.5, 1e6), (2.0, 3.3)):
        T = pgg.threshold_table(r, K)
        for sx in (0, 1):
            for Sx in range(26):
                for Sy in range(26):
                    want = o.threshold(o.payoff_total(sx, Sx, r), o.payoff_total(1 - sx, Sy, r), K)
                    assert int(T[sx, Sx, Sy]) == want, (r, K, sx, Sx, Sy)
    for pay, K in (((1.0, 0.0, 1.04, 0.0), 0.1), ((1.0, 0.5, 1.5, 0.0), 0.5), ((3.0, -1.0, 5.0, 0.5), 2.0),
                   ((1.0, 0.0, 1.5, 0.0), 1e-6), ((2.0, 2.0, 2.0, 2.0), 0.4)):
        T = pgg.threshold_table(4.0, K, "pairwise", pay).reshape(-1)
        assert not T[50:].any()
        for sx in (0, 1):
            for nx in range(5):
                for ny in range(5):
                    want = o.threshold(o.pair_payoff_total(sx, nx, pay), o.pair_payoff_total(1 - sx, ny, pay), K)
                    assert int(T[(sx * 5 + nx) * 5 + ny]) == want, (pay, K, sx, nx, ny)


def test_host_threshold_table_argument_checks(lib):
    from paper_1704_08098_gb300 import pgg
    out = (ctypes.c_uint32 * (2 * 26 * 26))()
    assert lib.pgg_threshold_table(pgg.GAME_GROUP, 4.0, 0.5, None, None) == pgg.PGG_ERR_ARG
    assert lib.pgg_threshold_table(pgg.GAME_GROUP, 4.0, 0.0, None, out) == pgg.PGG_ERR_ARG
    assert lib.pgg_threshold_table(pgg.GAME_GROUP, -1.0, 0.5, None, out) == pgg.PGG_ERR_ARG
    assert lib.pgg_threshold_table(pgg.GAME_PAIRWISE, 4.0, 0.5, None, out) == pgg.PGG_ERR_ARG
    assert lib.pgg_threshold_table(7, 4.0, 0.5, None, out) == pgg.PGG_ERR_ARG
    assert lib.pgg_threshold_table(pgg.GAME_GROUP, 4.0, 0.5, None, out) == pgg.PGG_OK


def test_stored_bench_line_keeps_the_contract():
    """The committed bench line (results/) carries the keys of the benchmark contract, and its
    figures agree with each other: value = L^2 site updates per step / the mean step time,
    roofline.frac = achieved / peak, the HBM figure = bytes per update x rate / peak."""
    import json
    d = json.load(open(os.path.join(ROOT, "results", "bench_L8192_bitpack_default.json")))
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert k in d, k
    L = d["config"]["L"]
    assert abs(d["value"] - L * L / (d["ms_per_step"] / 1e3)) <= 1e-6 * d["value"]
    r = d["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in r, k
    assert abs(r["frac"] - r["achieved"] / r["peak"]) <= 1e-9
    assert abs(r["hbm_frac"] - r["hbm_bytes_per_update"] * d["value"] / 1e9 / r["hbm_model"]["peak_gbs"]) <= 1e-6
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] > 0 and cb["sample"]
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] == L * L // 8 and e["d2h_bytes_per_step"] == 8
    assert d["gpu_launches"] >= d["steps"]
    assert not set(d["clocks"]["reasons"]) & {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}
