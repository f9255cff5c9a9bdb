"""The allocation-free entry point's source names no allocating call: no
cudaMalloc family, no stream-ordered pool, none of the library's own
allocation helpers (which route to a caller's allocator).  Runs on the CPU."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_1901_10026_gb300", "csrc", "tg_noalloc.cu")


def test_noalloc_source_names_no_allocation():
    text = open(SRC).read()
    code = re.sub(r"//[^\n]*", "", text)  # comments may describe what is not done
    for name in ("cudaMalloc", "cudaFree", "cudaMallocAsync", "cudaFreeAsync", "cudaMemPool",
                 "cudaMallocManaged", "cudaMallocHost", "cudaHostAlloc", "tg_dalloc", "tg_dfree",
                 "DevBuf", "malloc(", "new "):
        assert name not in code, name
