"""Every kernel launch passes its kernel's compile-time block size.

The kernels index shared arrays, digits, warps and tile rows by thread; a
launch with fewer threads than the kernel was written for leaves parts of that
state unwritten (a radix-sort histogram launched with half its digit threads
once produced scatter positions outside the output and a GPU memory fault).
Each kernel therefore declares its block size as the first argument of
__launch_bounds__, and this test (no GPU needed) parses the CUDA sources and
checks that every <<<grid, block>>> launch of that kernel names exactly the
same constant, and that every kernel declares one.
"""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2604_01397_b300", "csrc")


def _balanced(s: str, i: int) -> int:
    """Index just past the parenthesis group that opens at s[i]."""
    depth = 0
    for j in range(i, len(s)):
        if s[j] == "(":
            depth += 1
        elif s[j] == ")":
            depth -= 1
            if depth == 0:
                return j + 1
    raise AssertionError("unbalanced parentheses")


def _split_top(args: str):
    out, depth, cur = [], 0, ""
    for ch in args:
        if ch in "([":
            depth += 1
        elif ch in ")]":
            depth -= 1
        if ch == "," and depth == 0:
            out.append(cur.strip())
            cur = ""
        else:
            cur += ch
    out.append(cur.strip())
    return out


def _kernels(src: str):
    out = {}
    for m in re.finditer(r"__global__\s+void\s+", src):
        rest = src[m.end():]
        if rest.startswith("__launch_bounds__"):
            i = rest.index("(")
            j = _balanced(rest, i)
            nt = _split_top(rest[i + 1:j - 1])[0]
            name = re.match(r"\s*(\w+)\s*\(", rest[j:]).group(1)
        else:
            name = re.match(r"(\w+)\s*\(", rest).group(1)
            nt = None
        out[name] = nt
    return out


def _launches(src: str):
    for m in re.finditer(r"(\w+)\s*(<[^<>;]*>)?\s*<<<(.*?)>>>", src, flags=re.S):
        yield m.group(1), _split_top(m.group(3))


def test_every_launch_uses_its_kernels_block_size():
    srcs = {os.path.basename(p): open(p).read() for p in glob.glob(os.path.join(CSRC, "*.cu"))}
    kernels = {}
    for name, src in srcs.items():
        for k, nt in _kernels(src).items():
            assert nt is not None, f"{name}: kernel {k} declares no __launch_bounds__ block size"
            kernels[k] = nt
    assert len(kernels) >= 20
    seen = 0
    for name, src in srcs.items():
        for k, cfg in _launches(src):
            assert k in kernels, f"{name}: launch of unknown kernel {k}"
            assert len(cfg) >= 2, f"{name}: launch of {k} without a block size"
            assert re.sub(r"\s+", "", cfg[1]) == re.sub(r"\s+", "", kernels[k]), \
                f"{name}: {k} launched with block {cfg[1]!r}, declared {kernels[k]!r}"
            seen += 1
    assert seen >= 30
