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


def _sources():
    for path in glob.glob(os.path.join(CSRC, "*.cu*")) + glob.glob(os.path.join(CSRC, "*.h")):
        yield path, re.sub(r"//.*", "", open(path).read())


def test_no_device_traps_or_asserts():
    """Failures are reported through status words, never by trapping the GPU."""
    for path, text in _sources():
        for pat in (r"__trap\s*\(", r"\btrap\s*;", r"\bassert\s*\(", r"__brkpt\s*\("):
            assert not re.search(pat, text), (path, pat)


def test_no_cluster_multicast_copies():
    """Tiles are staged per CTA; no multicast TMA, so the code stays safe to run beside other ranks."""
    for path, text in _sources():
        assert ".multicast::cluster" not in text, path


def test_no_device_setting_changes():
    """Nothing changes clocks, power limits or other persistent GPU settings, or resets the device."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    files = glob.glob(os.path.join(CSRC, "*")) + glob.glob(os.path.join(root, "*.py")) + \
        glob.glob(os.path.join(root, "paper_2609_16863_gb300", "*.py"))
    for path in files:
        if os.path.isdir(path):
            continue
        text = open(path, errors="replace").read()
        for pat in (r"nvmlDeviceSet\w*", r"cudaDeviceReset\s*\(", r"nvidia-smi\s+-(lgc|rgc|ac|pl|pm)\b"):
            assert not re.search(pat, text), (path, pat)
