"""The resident-A complex64 update's tile schedule (csrc/gf_ra_sched.h, the same header the
kernel includes), compiled for the host with g++: for every CTA of the grid its runs of column
tiles, checked to cover every (row tile, column tile) exactly once, with the balance and the
number of runs (A loads) the schedule is designed for."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2202_05388_gb300", "csrc")

HARNESS = r'''
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "gf_ra_sched.h"
int main(int argc, char** argv) {
  const int64_t nrt = atoll(argv[1]), nct = atoll(argv[2]), G = atoll(argv[3]);
  std::vector<unsigned char> seen((size_t)(nrt * nct), 0);
  int64_t dup = 0, bad = 0, maxt = 0, mint = -1, maxruns = 0, total = 0;
  for (int64_t b = 0; b < G; ++b) {
    gf::RaCursor k;
    int64_t t = 0, runs = 0;
    for (bool more = gf::ra_first(k, nrt, nct, G, b); more; more = gf::ra_next(k, nrt, nct, G, b)) {
      if (k.rt < 0 || k.rt >= nrt || k.c < 0 || k.c >= nct || k.c < k.cbeg || k.c >= k.cend || k.cend > nct) { ++bad; break; }
      if (k.c == k.cbeg) ++runs;
      unsigned char& s = seen[(size_t)(k.rt * nct + k.c)];
      if (s) ++dup;
      s = 1;
      ++t;
    }
    total += t;
    if (t > maxt) maxt = t;
    if (mint < 0 || t < mint) mint = t;
    if (runs > maxruns) maxruns = runs;
  }
  int64_t missing = 0;
  for (unsigned char s : seen) missing += s ? 0 : 1;
  printf("%lld %lld %lld %lld %lld %lld %lld\n", (long long)total, (long long)dup, (long long)missing,
         (long long)bad, (long long)maxt, (long long)mint, (long long)maxruns);
  return 0;
}
'''


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("ra_sched")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    exe = d / "h"
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    return str(exe)


def _run(exe, nrt, nct, G):
    out = subprocess.run([exe, str(nrt), str(nct), str(G)], check=True, capture_output=True, text=True).stdout
    total, dup, missing, bad, maxt, mint, maxruns = map(int, out.split())
    return dict(total=total, dup=dup, missing=missing, bad=bad, maxt=maxt, mint=mint, maxruns=maxruns)


# (row tiles, column tiles, CTAs, smallest balance ideal/max, most runs per CTA)
CASES = [
    (801, 1601, 152, 0.98, 6),     # 320x320 workload (n = 102401)
    (1351, 2701, 152, 0.98, 9),    # 3-D lens 120x120x4 (n = 172803)
    (362, 723, 152, 0.95, 3),      # 215x215: two full groups + a last group in two segments per row
    (97, 193, 152, 0.99, 2),       # 3-D 32x32x4: one partial group, contiguous ranges
    (257, 513, 152, 0.99, 3),      # 512x64 (n = 32769)
    (16, 32, 152, 0.84, 2), (40, 79, 152, 0.985, 2), (129, 257, 152, 0.99, 2), (153, 305, 152, 0.99, 2),
    (1, 1, 1, 1.0, 1), (1, 300, 152, 0.98, 1), (300, 1, 152, 0.98, 2), (3, 5, 15, 1.0, 1), (2, 3, 6, 1.0, 1),
]


@pytest.mark.parametrize("nrt,nct,G,balance,runs", CASES)
def test_every_tile_exactly_once(harness, nrt, nct, G, balance, runs):
    G = min(G, nrt * nct)                      # the launch's grid: at most one CTA per tile
    r = _run(harness, nrt, nct, G)
    assert r["bad"] == 0 and r["dup"] == 0 and r["missing"] == 0
    assert r["total"] == nrt * nct
    assert (nrt * nct / G) / r["maxt"] >= balance, r
    assert r["maxruns"] <= runs, r
