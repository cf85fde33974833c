"""The pointer rule of the allocation-free entry point, on the CPU: a buffer
is accepted when it is device memory of the current device or managed
memory; host memory, unregistered memory and device memory of another GPU
are rejected. The rule's own header is compiled with g++ against the CUDA
runtime's declarations (no GPU and no CUDA library call needed)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2212_01317_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"


def test_pointer_rule(tmp_path):
    if shutil.which("g++") is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime_api.h")):
        pytest.skip("g++ or the CUDA headers are missing")
    src = tmp_path / "rule.cpp"
    src.write_text(r'''
#include <cstdio>
#include "mpr_ptrcheck.h"
int main() {
  using mpr::noalloc_pointer_ok;
  int bad = 0;
  bad += !noalloc_pointer_ok(cudaMemoryTypeDevice, 0, 0);
  bad += !noalloc_pointer_ok(cudaMemoryTypeDevice, 3, 3);
  bad += noalloc_pointer_ok(cudaMemoryTypeDevice, 1, 0);     /* another GPU's memory */
  bad += noalloc_pointer_ok(cudaMemoryTypeDevice, 0, 5);
  bad += !noalloc_pointer_ok(cudaMemoryTypeManaged, 2, 0);
  bad += noalloc_pointer_ok(cudaMemoryTypeHost, 0, 0);
  bad += noalloc_pointer_ok(cudaMemoryTypeUnregistered, 0, 0);
  std::printf("%d\n", bad);
  return bad;
}
''')
    exe = tmp_path / "rule"
    subprocess.run(["g++", "-std=c++17", "-I", CSRC, "-I", CUDA_INC, str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout
