"""The compression server's device-memory arena bookkeeping (host code,
csrc/atdct16_arena.h) against a brute-force granule map: first fit, no
overlap, exact accounting and full coalescing, over a long random sequence
of allocations and releases.  No GPU needed."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

HARNESS = r"""
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "atdct16_arena.h"

int main() {
  const size_t kGran = 256, kSize = 4u << 20, kN = kSize / kGran;
  atdct16::Arena a;
  a.init(kSize);
  std::vector<char> used(kN, 0);  // brute-force model, one flag per granule
  struct Live { size_t off, bytes; };
  std::vector<Live> live;
  std::mt19937_64 rng(1606);
  size_t model_used = 0;
  for (int step = 0; step < 20000; ++step) {
    if (live.empty() || rng() % 100 < 55) {
      const size_t bytes = 1 + rng() % (64u << 10);
      const size_t n = (bytes + kGran - 1) / kGran;
      // model: lowest start of a free run of n granules
      size_t best = kN, run = 0;
      for (size_t g = 0; g < kN; ++g) {
        run = used[g] ? 0 : run + 1;
        if (run == n) { best = g + 1 - n; break; }
      }
      size_t off = 0;
      const bool ok = a.alloc(bytes, &off);
      if (ok != (best < kN)) { std::printf("fail alloc-result step %d\n", step); return 1; }
      if (!ok) continue;
      if (off != best * kGran) { std::printf("fail first-fit step %d %zu %zu\n", step, off, best * kGran); return 1; }
      for (size_t g = best; g < best + n; ++g) used[g] = 1;
      live.push_back({off, bytes});
      model_used += n * kGran;
    } else {
      const size_t k = rng() % live.size();
      a.release(live[k].off, live[k].bytes);
      const size_t n = (live[k].bytes + kGran - 1) / kGran;
      for (size_t g = live[k].off / kGran; g < live[k].off / kGran + n; ++g) used[g] = 0;
      model_used -= n * kGran;
      live[k] = live.back();
      live.pop_back();
    }
    if (a.used() != model_used) { std::printf("fail accounting step %d\n", step); return 1; }
  }
  for (const Live& l : live) a.release(l.off, l.bytes);
  size_t off = 1;
  if (a.used() != 0 || !a.alloc(kSize, &off) || off != 0) { std::printf("fail coalescing\n"); return 1; }
  std::printf("ok\n");
  return 0;
}
"""


def test_arena_first_fit_accounting_and_coalescing(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    src, exe = tmp_path / "arena.cpp", tmp_path / "arena"
    src.write_text(HARNESS)
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "paper_1606_05562_gb300", "csrc"),
                    str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout
