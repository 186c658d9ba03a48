// Tile schedule of the resident-A complex64 update (k_rank_update_c64_ra): which (row tile,
// column tile) pairs CTA b of G visits, in runs that share one row tile (one load of its A
// blocks per run).  Plain integer arithmetic, compiled for the device by nvcc and for the host by
// the CPU tests, which check that every tile is visited exactly once.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define GF_RA_FN __host__ __device__ __forceinline__
#else
#define GF_RA_FN inline
#endif

namespace gf {

struct RaCursor {
  int64_t g, rt, c, cbeg, cend;
  int64_t lnext, lend;                          // rest of a contiguous range in its group
};
// Runs of CTA b of G.  A group of R row tiles (R = G except in the last group) is split into s =
// G / R column segments per row tile when that keeps every CTA busy, or at least 3/4 of them where
// the B blocks of all column tiles would not stay in L2 (more than 512 column tiles); otherwise
// each CTA takes an equal contiguous range of the group's tiles in row-major order, a run per row
// tile it touches (the CTAs then read B blocks of different columns at any one time).
GF_RA_FN bool ra_piece(RaCursor& k, int64_t nct, int64_t G) {
  k.rt = k.g * G + k.lnext / nct;
  k.c = k.cbeg = k.lnext % nct;
  k.cend = (k.cbeg + (k.lend - k.lnext)) < nct ? (k.cbeg + (k.lend - k.lnext)) : nct;
  k.lnext += k.cend - k.cbeg;
  return true;
}
GF_RA_FN bool ra_run(RaCursor& k, int64_t nrt, int64_t nct, int64_t G, int64_t b) {
  for (; k.g * G < nrt; ++k.g) {
    const int64_t R = (nrt - k.g * G) < G ? (nrt - k.g * G) : G;
    const int64_t s = G / R;                  // column segments per row tile
    if (R * s == G || (nct > 512 && 4 * R * s >= 3 * G)) {
      if (b >= R * s) continue;
      const int64_t seg = b / R;
      const int64_t c0 = seg * nct / s, c1 = (seg + 1) * nct / s;
      if (c1 <= c0) continue;
      k.rt = k.g * G + b % R;
      k.c = k.cbeg = c0;
      k.cend = c1;
      k.lnext = k.lend = 0;
      return true;
    }
    const int64_t l0 = b * R * nct / G, l1 = (b + 1) * R * nct / G;
    if (l1 <= l0) continue;
    k.lnext = l0;
    k.lend = l1;
    return ra_piece(k, nct, G);
  }
  return false;
}
GF_RA_FN bool ra_first(RaCursor& k, int64_t nrt, int64_t nct, int64_t G, int64_t b) {
  k.g = 0;
  return ra_run(k, nrt, nct, G, b);
}
GF_RA_FN bool ra_next(RaCursor& k, int64_t nrt, int64_t nct, int64_t G, int64_t b) {
  if (++k.c < k.cend) return true;
  if (k.lnext < k.lend) return ra_piece(k, nct, G);
  ++k.g;
  return ra_run(k, nrt, nct, G, b);
}

}  // namespace gf
