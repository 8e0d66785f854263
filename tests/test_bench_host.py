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
