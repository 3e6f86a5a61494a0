"""The pool's arena allocator (csrc/gp_arena.h, host code) against a brute-force model
of the arena on the CPU: random allocations and releases; every allocation is the
lowest aligned gap that fits (first fit), allocations never overlap or leave the
arena, the free bytes and the largest free block match the model, and releasing
everything coalesces the arena back into one block."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1605_03958_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include <map>
#include <random>
#include <vector>
#include "gp_arena.h"

using gp_arena::Arena;
using gp_arena::kArenaAlign;

// the model: the live allocations (offset -> aligned size) of an arena of cap bytes
struct Model {
  size_t cap;
  std::map<size_t, size_t> live;
  // lowest offset of a free gap of at least b bytes, or cap if none
  size_t first_fit(size_t b) const {
    size_t at = 0;
    for (const auto& a : live) {
      if (a.first - at >= b) return at;
      at = a.first + a.second;
    }
    return cap - at >= b ? at : cap;
  }
  size_t free_total() const {
    size_t used = 0;
    for (const auto& a : live) used += a.second;
    return cap - used;
  }
  size_t largest() const {
    size_t at = 0, m = 0;
    for (const auto& a : live) {
      m = std::max(m, a.first - at);
      at = a.first + a.second;
    }
    return std::max(m, cap - at);
  }
};

#define CHECK(c) do { if (!(c)) { std::printf("FAIL line %d: %s\n", __LINE__, #c); return 1; } } while (0)

int main() {
  std::mt19937_64 rng(1605);
  for (int trial = 0; trial < 40; ++trial) {
    const size_t cap = kArenaAlign * (1 + rng() % 4000);
    Arena A;
    A.reset(cap);
    Model M{cap, {}};
    std::vector<std::pair<size_t, size_t>> held;   // (offset, requested bytes)
    for (int op = 0; op < 3000; ++op) {
      if (held.empty() || rng() % 100 < 55) {
        const size_t req = 1 + rng() % (cap / 8 + 1);
        const size_t b = gp_arena::align_up(req, kArenaAlign);
        size_t off = 0;
        const bool ok = A.alloc(req, &off);
        const size_t want = M.first_fit(b);
        CHECK(ok == (want < cap));
        if (ok) {
          CHECK(off == want);
          CHECK(off % kArenaAlign == 0 && off + b <= cap);
          M.live[off] = b;
          held.push_back({off, req});
        }
      } else {
        const size_t k = rng() % held.size();
        A.release(held[k].first, held[k].second);
        M.live.erase(held[k].first);
        held.erase(held.begin() + k);
      }
      CHECK(A.free_total() == M.free_total());
      CHECK(A.largest() == M.largest());
    }
    for (const auto& h : held) A.release(h.first, h.second);
    CHECK(A.free_total() == cap && A.largest() == cap && A.high_water() == 0);
    size_t off = 1;
    CHECK(A.alloc(cap, &off) && off == 0);   // one block again: the whole arena fits
    CHECK(!A.alloc(1, &off));
  }
  std::printf("ok\n");
  return 0;
}
"""


def test_arena_first_fit_and_coalescing(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "arena_driver.cpp"
    exe = tmp_path / "arena_driver"
    src.write_text(DRIVER)
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
