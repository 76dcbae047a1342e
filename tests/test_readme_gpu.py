"""The usage example of README.md runs as written and gives sensible output."""
import os
import re

import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_python_example_runs():
    text = open(os.path.join(ROOT, "README.md")).read()
    block = re.search(r"```python\n(.*?)```", text, re.S).group(1)
    env = {}
    exec(compile(block, "README.md", "exec"), env)
    rho, mu, Hk = env["rho"], env["mu"], env["Hk"]
    assert abs(mu[0].item() - 1.0) < 1e-12                   # +-1 vectors: mu_0 = 1
    assert torch.isfinite(rho).all() and (rho > -1e-3).all()  # Jackson damping keeps the DOS ~ >= 0
    assert Hk.dtype == torch.complex128 and Hk.get_values().abs().sum().item() > 0
