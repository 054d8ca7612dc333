"""bench.py reports a kernel's captured DRAM traffic only while the kernel is unchanged: the
key is a hash of the kernel's definition and of the device helpers it calls. Every helper
the kernel calls (transitively, within its source file) must be part of that key, or a
change to the helper would leave a stale traffic figure in place."""
import re
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
sys.path.insert(0, str(ROOT))
import bench  # noqa: E402

CSRC = ROOT / "paper_1404_3816_gb300" / "csrc"


def _called_helpers(text, name, seen):
    body = bench._definition(text, name)
    # device functions of the file (double-underscore names are CUDA attributes and built-ins)
    defined = {d for d in re.findall(r"__device__[^(;{]*?\b([A-Za-z_]\w*)\s*\(", text) if not d.startswith("__")}
    for c in set(re.findall(r"\b([A-Za-z_]\w*)\s*[<(]", body)):
        if c in defined and c != name and c not in seen:
            seen.add(c)
            _called_helpers(text, c, seen)
    return seen


@pytest.mark.parametrize("kind", sorted(bench.KERNEL_SOURCES))
def test_traffic_key_covers_the_kernel_and_its_helpers(kind):
    f, names, _ = bench.KERNEL_SOURCES[kind]
    text = (CSRC / f).read_text()
    assert bench._definition(text, names[0]), f"{names[0]} not found in {f}"
    for nm in names:
        assert bench._definition(text, nm), f"{nm} listed for {kind} but not defined in {f}"
    missing = sorted(_called_helpers(text, names[0], set()) - set(names))
    assert not missing, f"{kind}: helpers called by {names[0]} but not hashed: {missing}"
