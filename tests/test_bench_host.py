"""Host-side logic of bench.py (CPU): the step kernel's source hash that keys
the recorded DRAM traffic, and the algorithmic byte counts."""
import bench


def test_function_text_includes_declaration_and_template():
    src = ("// note\n"
           "template <int U>\n"
           "__global__ void __launch_bounds__(1024, 2) walk_f64(Args a) {\n"
           "    if (a.n) { body(); }\n"
           "}\n"
           "int other() { return 1; }\n")
    t = bench._function_text(src, "walk_f64(Args a)")
    assert t.startswith("template <int U>\n__global__ void __launch_bounds__(1024, 2) walk_f64")
    assert t.endswith("}") and "other" not in t
    # a changed compile hint changes the text, hence the hash key
    t2 = bench._function_text(src.replace("(1024, 2)", "(1024)"), "walk_f64(Args a)")
    assert t2 != t


def test_step_hash_covers_every_step_function():
    import os
    src = open(os.path.join(bench.ROOT, "paper_0910_4836_gb300", "csrc", "jds.cu")).read()
    fam = bench.STEP_FUNCTIONS["SELL"]
    for sig in fam[1]:
        assert sig in src, sig  # each hashed function still exists
        assert bench._function_text(src, sig)
    h = bench.kernel_source_hash("SELL row_only w=128 u=4")
    assert len(h) == 12 and h == bench.kernel_source_hash("SELL row_only w=1024 u=4")


def test_algorithmic_bytes():
    # val + col once, row_ptr once, x at least once, y once
    assert bench.algorithmic_bytes(10, 20, 100) == 8 * 100 + 4 * 100 + 4 * 11 + 8 * 20 + 8 * 10
    assert bench.algorithmic_bytes(10, 20, 100, vbytes=4) == 4 * 100 + 4 * 100 + 4 * 11 + 4 * 20 + 4 * 10


def test_reference_arm_line_contract(monkeypatch):
    """--impl reference times the CPU oracle and prints the contract's keys
    (here on the small Laplacian workload, rank 0 of one)."""
    import argparse
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    args = argparse.Namespace(config=0, steps=3, warmup=1)
    r = bench.run_reference(args)
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "impl", "config", "cpu_baseline", "e2e"):
        assert key in r, key
    assert r["impl"] == "reference" and r["value"] > 0 and r["steps"] == 3 and r["higher_is_better"] is True
    assert r["config"]["workload"].startswith("laplace2d") and r["config"]["n_rows"] == 4096
    cb = r["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == r["value"] and cb["cores"] >= 1 and cb["sample"]
    assert r["e2e"] == {"value": r["value"], "unit": r["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # other ranks print nothing
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(args) is None


def test_method_bytes_and_basis_labels():
    """The JDS family's method bytes (val + col, the pointer array, x once,
    y once) leave out the format's own arrays; every credited form names one
    basis for both vectors."""
    class A:
        nnz, n_rows, n_cols = 100, 10, 20
    assert bench.jds_method_bytes(A, 4) == 12 * 100 + 4 * 4 + 8 * 20 + 8 * 10
    c = bench.Cand("x", None, None, "mixed", 1, credited=False)
    assert not c.credited and "NOT one basis" in bench.BASIS_LABEL["mixed"]
    assert set(bench.BASIS_LABEL) == {"original", "permuted", "mixed"}
