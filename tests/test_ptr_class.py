"""Pointer classification of the C ABI (CPU only): every entry point takes host or device arrays
and must refuse an array in another GPU's memory (its kernels run on the current device, where
such a pointer is an illegal address).  The decision is a pure function of the pointer's CUDA
attributes and the current device; it is compiled here with the host compiler and checked on
made-up attributes, so no GPU and no kernel is involved."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2304_07325_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

PROG = r"""
#include <cstdio>
#include "ptr_class.h"
int main() {
  struct { cudaMemoryType t; int owner, cur, want; } cases[] = {
    {cudaMemoryTypeDevice, 0, 0, PTR_DEVICE},        // this GPU's memory: used in place
    {cudaMemoryTypeDevice, 3, 3, PTR_DEVICE},
    {cudaMemoryTypeDevice, 1, 0, PTR_FOREIGN},       // another GPU's memory: refused
    {cudaMemoryTypeDevice, 0, 5, PTR_FOREIGN},
    {cudaMemoryTypeManaged, 2, 0, PTR_DEVICE},       // managed memory: any device may touch it
    {cudaMemoryTypeHost, 1, 0, PTR_HOST},            // page-locked host memory: copied
    {cudaMemoryTypeUnregistered, 0, 0, PTR_HOST},    // plain host memory: copied
  };
  int bad = 0;
  for (auto &c : cases) {
    int got = classify_pointer(c.t, c.owner, c.cur);
    if (got != c.want) { std::printf("type %d owner %d current %d: %d, want %d\n", (int)c.t, c.owner, c.cur, got, c.want); ++bad; }
  }
  std::printf("%d bad\n", bad);
  return bad;
}
"""


@pytest.mark.skipif(shutil.which("g++") is None or not os.path.isdir(CUDA_INC), reason="needs g++ and the CUDA headers")
def test_foreign_device_pointers_are_refused(tmp_path):
    src = tmp_path / "ptr_class_check.cpp"
    src.write_text(PROG)
    exe = tmp_path / "ptr_class_check"
    # the header is host code over the runtime's types; linking needs no CUDA library because
    # only classify_pointer (pure) is called
    subprocess.check_call(["g++", "-std=c++17", "-O1", f"-I{CSRC}", f"-I{CUDA_INC}", str(src), "-o", str(exe),
                           "-Wl,--unresolved-symbols=ignore-all"])
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("0 bad")


def test_every_entry_point_classifies_through_the_shared_helper():
    """The host-side staging (api.cu) and the allocation-free entry point (k_static.cu) both
    decide through pointer_class, so neither can accept another GPU's array."""
    api = open(os.path.join(CSRC, "api.cu")).read()
    st = open(os.path.join(CSRC, "k_static.cu")).read()
    assert '#include "ptr_class.h"' in api and '#include "ptr_class.h"' in st
    assert "cudaPointerGetAttributes" not in api and "cudaPointerGetAttributes" not in st
    assert "pointer_class(src)" in api and "pointer_class(p) == PTR_DEVICE" in st
