"""Source check of the chained launches (programmatic dependent launch).

A kernel launched with launch_chained may be scheduled before the kernel
ahead of it in the stream has finished; it is correct only if it calls
chain_enter() (griddepcontrol.wait) before it touches global memory.  This
test reads the CUDA sources and checks that every kernel that can reach a
launch_chained call, directly or through an `auto` variable that selects
between instantiations, has chain_enter() as the first statement of its
body.  No GPU is needed."""
import glob
import os
import re

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2311_16728_b300", "csrc")


def _sources():
    return {os.path.basename(p): open(p).read() for p in glob.glob(os.path.join(CSRC, "*.cu"))}


def _chained_kernels(src):
    """Kernel names launched by launch_chained in one source file."""
    names = set()
    for m in re.finditer(r"launch_chained\(\s*([A-Za-z_]\w*)", src):
        ident = m.group(1)
        if ident.endswith("_kernel"):
            names.add(ident)
            continue
        # an `auto ident = cond ? a_kernel<..> : b_kernel<..>;` before the call
        defs = list(re.finditer(r"auto\s+" + ident + r"\s*=\s*([^;]*);", src[:m.start()]))
        assert defs, f"launch_chained({ident}, ...): no definition of {ident} found"
        found = set(re.findall(r"\b(\w+_kernel)\b", defs[-1].group(1)))
        assert found, f"launch_chained({ident}, ...): {ident} names no kernel"
        names |= found
    return names


def _body_start(src, kernel):
    """The text of the kernel's body after its opening brace."""
    m = re.search(r"__global__\s+void[^;{]*?\b" + kernel + r"\s*\(", src, re.S)
    assert m, f"no definition of {kernel}"
    depth, i = 0, m.end() - 1
    while True:  # the parameter list's closing parenthesis
        depth += {"(": 1, ")": -1}.get(src[i], 0)
        if depth == 0:
            break
        i += 1
    return src[src.index("{", i) + 1:]


def test_every_chained_kernel_waits_first():
    srcs = _sources()
    chained = set()
    for src in srcs.values():
        chained |= _chained_kernels(src)
    assert {"render_fwd_warp_kernel", "render_bwd_warp_kernel", "adam_kernel", "ssim_pass1_kernel"} <= chained
    for kernel in sorted(chained):
        owner = [s for s in srcs.values() if re.search(r"__global__\s+void[^;{]*?\b" + kernel + r"\s*\(", s, re.S)]
        assert len(owner) == 1, f"{kernel}: defined in {len(owner)} files"
        body = _body_start(owner[0], kernel)
        first = re.sub(r"//[^\n]*", "", body).strip()
        assert first.startswith("chain_enter();"), f"{kernel} is launched chained but does not wait first"
