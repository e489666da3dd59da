"""The usage example of the README runs as written."""
import os
import re

import pytest

pytestmark = pytest.mark.gpu


def test_readme_example_runs():
    from tests.gpu_util import gpu_available
    if not gpu_available():
        pytest.skip("no CUDA device")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    text = open(os.path.join(root, "README.md")).read()
    blocks = re.findall(r"```python\n(.*?)```", text, re.S)
    assert len(blocks) == 1
    scope = {}
    exec(compile(blocks[0], "README example", "exec"), scope)
    assert (scope["cls"] == scope["wl"].labels).mean() > 0.9
    import numpy as np
    q = float(np.mean(scope["wl"].labels == 0))
    root_entropy = -(q * np.log(q) + (1 - q) * np.log(1 - q))
    assert scope["r"]["loss"] < root_entropy
    assert scope["q"]["valid"] and scope["q"]["loss"] < root_entropy
    loss = scope["boost"].train_loss
    assert len(loss) == 10 and np.all(np.diff(loss) <= 0)
    scope["tree"].free()
    scope["boost"].free()
    scope["ctx"].close()
