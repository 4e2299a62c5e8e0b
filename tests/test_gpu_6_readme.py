"""The README's code blocks run as written (in order, one namespace) on the GPU."""
import os
import re

import pytest
import torch

pytestmark = pytest.mark.gpu

README = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "README.md")


def test_readme_examples_run():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    blocks = re.findall(r"```python\n(.*?)```", open(README).read(), flags=re.S)
    assert len(blocks) >= 5
    ns = {}
    for b in blocks:
        exec(compile(b, README, "exec"), ns)
    torch.cuda.synchronize()
    # the gradient example produced gradients for every parameter group and every agent
    assert ns["theta"].grad is not None and torch.isfinite(ns["theta"].grad).all()
    assert ns["x0"].grad is not None and bool(torch.isfinite(ns["x0"].grad).all())
