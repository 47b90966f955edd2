"""No C++ exception crosses the C ABI: the guard every entry point runs its
body through turns an exception into SNC_ERR_OOM with a readable last error,
and passes a body's own status through.  Host code only (no GPU): a small
program compiled with g++ against the library's internal header and linked
to the built libsnc.so."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2306_09855_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <cstring>
#include <new>
#include <stdexcept>
#include "snc_internal.h"

int main() {
  snc_status s = snc::abi_guard([]() -> snc_status { throw std::bad_alloc(); });
  if (s != SNC_ERR_OOM) return 1;
  if (!std::strstr(snc_last_error(nullptr), "host resources exhausted")) return 2;
  s = snc::abi_guard([]() -> snc_status { throw std::runtime_error("thread start"); });
  if (s != SNC_ERR_OOM || !std::strstr(snc_last_error(nullptr), "thread start")) return 3;
  s = snc::abi_guard([]() -> snc_status { throw 7; });
  if (s != SNC_ERR_OOM || !std::strstr(snc_last_error(nullptr), "unknown exception")) return 4;
  s = snc::abi_guard([]() -> snc_status { return SNC_ERR_STATE; });
  if (s != SNC_ERR_STATE) return 5;
  s = snc::abi_guard([]() -> snc_status { return SNC_OK; });
  if (s != SNC_OK) return 6;
  std::puts("ok");
  return 0;
}
"""


def test_exceptions_become_status_codes(tmp_path):
    gxx = shutil.which("g++")
    cuda_inc = "/usr/local/cuda/include"
    if gxx is None or not os.path.isdir(cuda_inc):
        pytest.skip("needs g++ and the CUDA headers")
    from paper_2306_09855_gb300 import _build
    lib = _build.build()
    src = tmp_path / "guard.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "guard"
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", CSRC, "-I", cuda_inc, str(src), "-o", str(exe),
                    lib, "-Wl,-rpath," + os.path.dirname(lib)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.strip() == "ok"
