"""CPU check of the sources: every kernel launched with programmatic stream serialisation (launch_dependent) waits
for the grids before it (grid_dependency_wait) before its first memory access.  Such a grid may be scheduled while
the previous kernel on the stream is still writing, so a kernel without the wait would read stale data."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2307_12607_gb300", "csrc")


def sources():
    return {os.path.basename(f): open(f).read() for f in glob.glob(os.path.join(CSRC, "*.cu*"))}


def body_after(text, start):
    """The brace-delimited body that starts at the first '{' at or after start."""
    i = text.index("{", start)
    depth = 0
    for j in range(i, len(text)):
        depth += {"{": 1, "}": -1}.get(text[j], 0)
        if depth == 0:
            return text[i:j + 1]
    raise AssertionError("unbalanced braces")


def kernels_launched_dependently(src):
    """Kernel names referenced by the host functions that call launch_dependent."""
    names = set()
    for name, text in src.items():
        for m in re.finditer(r"\n(?:static\s+)?cudaError_t\s+\w+\s*\(", text):
            body = body_after(text, m.end())
            if "launch_dependent(" in body:
                names |= set(re.findall(r"\b(\w+_kernel)\b", body))
    return names


def kernel_body(src, kernel):
    for text in src.values():
        m = re.search(r"__global__\s+void\s+(?:__launch_bounds__\([^)]*\)\s+)?" + kernel + r"\s*\(", text)
        if m:
            return body_after(text, m.end())
    raise AssertionError(f"no definition of {kernel}")


def test_dependent_launches_cover_the_pipeline_head():
    names = kernels_launched_dependently(sources())
    assert {"bounds_kernel", "plan_kernel", "engine_kernel"} <= names


def test_every_dependently_launched_kernel_waits_first():
    src = sources()
    for kernel in sorted(kernels_launched_dependently(src)):
        body = kernel_body(src, kernel)
        assert "grid_dependency_wait();" in body, kernel
        wait = body.index("grid_dependency_wait();")
        # nothing before the wait reads or writes global memory: only the kernel's shared memory set-up and index
        # arithmetic (no pointer from the parameters is dereferenced before it)
        head = body[:wait]
        assert not re.search(r"__ldg|__ldcg|atomic\w*\(\s*(?!&s\.)|\bp\.\w+\[|\bep\.\w+\[", head), kernel
