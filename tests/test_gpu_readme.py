"""The Python usage example of README.md runs as written (on a GPU)."""
import os
import re

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_readme_python_example_runs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_7461_gb300 import build

    build.build()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    text = open(os.path.join(root, "README.md")).read()
    blocks = re.findall(r"```python\n(.*?)```", text, re.S)
    assert blocks, "README.md has no python example"
    env = {}
    exec(compile(blocks[0], "README.md", "exec"), env)
    assert len(env["r"]) == env["cnt"] > 0
    assert len(env["pairs"]) > 0
