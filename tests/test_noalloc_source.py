"""The allocation-free BVH build names no allocator on its path (source check, no GPU).

st_build_bvh_noalloc runs its own checks, then the radix-tree build the
allocating path shares (bvh_build: morton_order, k_hierarchy, boxes). This
reads those function bodies and the entry point's file and fails if any of them
calls an allocator, so a later edit that adds one to the shared path cannot
pass unnoticed.
"""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2012_03939_gb300", "csrc")
ALLOC = re.compile(r"\b(cudaMalloc\w*|cudaHostAlloc|cudaMallocManaged|dalloc|malloc|calloc|realloc|"
                   r"cudaMemPool\w*|cuMem\w*Alloc\w*)\s*\(|\bnew\s+[A-Za-z_]")


def _body(src, signature):
    i = src.index(signature)
    j = src.index("{", i)
    depth = 0
    for k in range(j, len(src)):
        depth += {"{": 1, "}": -1}.get(src[k], 0)
        if depth == 0:
            return src[j:k + 1]
    raise AssertionError("unbalanced braces after " + signature)


def _strip_comments(src):
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return re.sub(r"//[^\n]*", "", src)


def test_noalloc_entry_point_file_calls_no_allocator():
    src = _strip_comments(open(os.path.join(CSRC, "st_noalloc.cu")).read())
    found = ALLOC.findall(src)
    assert not found, found


def test_shared_build_path_calls_no_allocator():
    src = _strip_comments(open(os.path.join(CSRC, "st_bvh.cu")).read())
    for sig in ("cudaError_t bvh_build(st_scene* s, cudaStream_t stream)",
                "cudaError_t morton_order(st_scene* s, cudaStream_t stream)",
                "cudaError_t boxes(st_scene* s, cudaStream_t stream)"):
        body = _body(src, sig)
        assert not ALLOC.search(body), (sig, ALLOC.findall(body))
    # the path calls only these host functions and kernels
    calls = set(re.findall(r"\b(k_\w+|morton_order|boxes)\s*<<<|\b(morton_order|boxes)\s*\(",
                           _body(src, "cudaError_t bvh_build(st_scene* s, cudaStream_t stream)")))
    assert calls, "the build body was not found"


def test_scan_catches_a_planted_allocation():
    planted = "cudaError_t boxes(st_scene* s, cudaStream_t stream) { char* b; cudaMalloc((void**)&b, 16); }"
    assert ALLOC.search(_body(planted, "cudaError_t boxes(st_scene* s, cudaStream_t stream)"))
