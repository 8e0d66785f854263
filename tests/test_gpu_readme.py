"""The README's Python example runs as written (guards the documented API)."""
import os
import re

import pytest

pytestmark = pytest.mark.gpu


def test_readme_example_runs():
    import paper_0910_4836_gb300 as g
    g.build()
    text = open(os.path.join(os.path.dirname(os.path.dirname(__file__)), "README.md")).read()
    code = re.search(r"```python\n(.*?)```", text, re.S).group(1)
    ns = {}
    exec(compile(code, "README.md", "exec"), ns)
    assert ns["loss"].item() > 0 and ns["val"].grad is not None and ns["Y"].shape[1] == 16
