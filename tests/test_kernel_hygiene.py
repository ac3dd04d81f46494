"""Every kernel of the library is launched with programmatic stream serialisation,
so every __global__ function must start with pdl_prologue() (wait for the previous
grid before touching memory).  A kernel without it would race its predecessor."""
import glob
import os
import re

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2609_16863_gb300", "csrc")


def test_every_kernel_starts_with_the_pdl_prologue():
    missing = []
    for path in glob.glob(os.path.join(CSRC, "*.cu*")):
        text = open(path).read()
        for m in re.finditer(r"__global__[^;{]*?\b(\w+)\s*\([^;{]*?\)\s*\{", text, flags=re.S):
            body = text[m.end(): m.end() + 200].lstrip()
            if not body.startswith("pdl_prologue();"):
                missing.append(f"{os.path.basename(path)}:{m.group(1)}")
    assert not missing, missing


def test_kernels_are_launched_through_launch():
    # a raw <<<...>>> launch would bypass the launch counter and the PDL attribute
    for path in glob.glob(os.path.join(CSRC, "*.cu*")):
        text = open(path).read()
        text = re.sub(r"//.*", "", text)
        lines = [ln for ln in text.splitlines() if "<<<" in ln and "k<<<grid" not in ln]
        assert not lines, (path, lines)
