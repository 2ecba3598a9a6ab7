"""Host logic: the per-context cache of library-owned streams and events (csrc/context_cache.h),
compiled with g++ and driven with made-up context ids.  A device reset gives the primary
context a new id, so the next call must make fresh objects rather than reuse the old handles;
the same (context, device) pair must keep its objects."""
import os
import shutil
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2104_05877_gb300", "csrc")

SOURCE = r"""
#include <cstdio>
#include "context_cache.h"

struct Obj { int serial = 0; };

#define CHECK(c) do { if (!(c)) { std::printf("FAIL line %d: %s\n", __LINE__, #c); return 1; } } while (0)

int main() {
  skel::ContextCache<Obj, 4> cache;
  int made = 0;
  auto make = [&](Obj& o) { o.serial = ++made; return true; };
  Obj* a = cache.get(7, 0, make);
  CHECK(a && a->serial == 1 && made == 1);
  CHECK(cache.get(7, 0, make) == a && made == 1);          // same context and device: kept
  Obj* b = cache.get(8, 0, make);                            // device reset: a new context id
  CHECK(b && b != a && b->serial == 2 && made == 2);
  Obj* c = cache.get(7, 1, make);                            // same id, another device
  CHECK(c && c != a && c != b && c->serial == 3);
  CHECK(cache.get(7, 0, make) == a && cache.get(8, 0, make) == b && made == 3);
  // a failed make caches nothing: the next call tries again
  auto fail = [&](Obj&) { ++made; return false; };
  CHECK(cache.get(9, 0, fail) == nullptr && made == 4);
  Obj* d = cache.get(9, 0, make);
  CHECK(d && d->serial == 5);
  // a fifth pair reuses the oldest slot (context 7, device 0), whose next lookup makes anew
  Obj* e = cache.get(10, 0, make);
  CHECK(e && e->serial == 6 && e == a);
  CHECK(cache.get(8, 0, make) == b && cache.get(7, 1, make) == c && cache.get(9, 0, make) == d);
  Obj* f = cache.get(7, 0, make);
  CHECK(f && f->serial == 7);
  // context id 0 (no ids offered by the driver) keys on the device alone
  Obj* g = cache.get(0, 2, make);
  CHECK(g && cache.get(0, 2, make) == g);
  std::printf("ok\n");
  return 0;
}
"""


def test_context_cache_keys_on_context_and_device(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    src = tmp_path / "check.cpp"
    src.write_text(SOURCE)
    exe = tmp_path / "check"
    r = subprocess.run([gxx, "-std=c++17", "-O1", "-Wall", "-Werror", "-I", CSRC, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
