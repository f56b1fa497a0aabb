"""Source invariants of the CUDA library that no numerical test would catch.

Every kernel is launched with programmatic stream serialization, so a kernel may start while the
kernel before it in the stream is still running; it is correct only because its first statement
waits for that kernel (griddepcontrol.wait, `pdl_wait()`).  These checks keep that true for every
kernel in `csrc/`, and keep every launch going through `launch_pdl`.
"""
import os
import re

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2111_02912_gb300", "csrc")


def _sources():
    for name in sorted(os.listdir(CSRC)):
        if name.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(CSRC, name)) as f:
                yield name, f.read()


def _strip_comments(text):
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return re.sub(r"//[^\n]*", "", text)


def test_every_kernel_waits_for_its_predecessor_first():
    kernels = 0
    for name, text in _sources():
        code = _strip_comments(text)
        for m in re.finditer(r"__global__\s+void[^{;]*?\b(\w+)\s*\([^)]*\)\s*\{", code):
            kernels += 1
            body = code[m.end():]
            first = body.lstrip().split(";", 1)[0].strip()
            assert first == "pdl_wait()", "%s: kernel %s starts with %r, not pdl_wait()" % (name, m.group(1), first)
    assert kernels >= 15


def test_no_kernel_is_launched_without_launch_pdl():
    for name, text in _sources():
        code = _strip_comments(text)
        assert "<<<" not in code, "%s launches a kernel with <<< >>> instead of launch_pdl" % name
