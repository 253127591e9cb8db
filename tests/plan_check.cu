// Host-only checks of the tensor-core work plan (no device work): built and run by
// tests/test_plan_host.py. It includes the library's host source, so that the
// planner's internal functions are in reach, and links the built library for the
// launchers that source refers to.
//
// Checked for every configuration:
//  * coverage: each (output row strip, output column) pair of the evaluated part is
//    in exactly one main work unit (upper triangle, Sec. 3.3: columns from the
//    strip's own first row on; both triangles: every column);
//  * list slots: a unit's row-side lists lie in its strip's slot range, and every
//    slot the merge reads for a strip's rows is written by exactly one unit;
//  * band units: one per strip, inside the series, covering the strip's own block;
//  * phases of a host-buffer call: the units of phase q evaluate only strips of that
//    phase and read only days from the phase's first day on, and phase 0 holds the
//    days the centring mean reads;
//  * the default work-unit length against the Gram tiles per SM.
// Prints one line per failure and exits non-zero if there was any.
#include "../paper_2603_02059_gb300/csrc/traknn_api.cu"

#include <cstdio>
#include <map>

namespace {

int g_fail = 0;

void fail(const char* what, int a, int b) {
  std::printf("FAIL %s (%d, %d)\n", what, a, b);
  ++g_fail;
}

void check_plan(int B, int64_t N0, int L, int tiles, int group, int egroups, int sym,
                int part_lo, int part_hi, const std::vector<int>& pstrip, int band_tiles) {
  std::vector<HostSeries> sd(B);
  for (int b = 0; b < B; ++b)
    sd[b] = HostSeries{nullptr, N0 - 97 * b, L + (b % 3), 10, L + (b % 3) - 1, nullptr, nullptr,
                       nullptr};
  TcPlan p;
  build_plan(sd.data(), B, 100, sym, 0, tiles, group, false, part_lo, part_hi, pstrip, egroups,
             band_tiles, p);
  if ((int)p.slot_lo.size() != (int)p.col_off.size()) fail("slot table size", 0, 0);
  for (int b = 0; b < B; ++b) {
    const SeriesInfo& si = p.table.s[b];
    const int M = si.M, R = si.rows_out, strips = (M + R - 1) / R;
    const int slo = std::max(0, part_lo), shi = std::min(strips, part_hi);
    std::vector<std::vector<int>> cover(strips);
    std::vector<std::map<int, int>> written(strips);
    for (int u = 0; u < p.nunits; ++u) {
      const WorkUnit& w = p.units[u];
      if (w.series != b) continue;
      if (w.strip < slo || w.strip >= shi) {
        fail("unit outside the evaluated strips", b, w.strip);
        continue;
      }
      std::vector<int>& c = cover[w.strip];
      if (c.empty()) c.assign(M, 0);
      for (int j = std::max(0, w.jlo); j < std::min(w.jhi, M); ++j) ++c[j];
      ++written[w.strip][w.slot];
      const int lo = p.slot_lo[si.strip_base + w.strip];
      if (w.slot * egroups < lo || (w.slot + 1) * egroups > si.slots) fail("slot range", b, u);
    }
    for (int s = slo; s < shi; ++s) {
      for (int j = 0; j < M; ++j) {
        const int want = (!sym || j >= s * R) ? 1 : 0;
        const int got = cover[s].empty() ? 0 : cover[s][j];
        if (got != want) {
          fail("column coverage", s, j);
          break;
        }
      }
      // the merge reads the slots [slot_lo, slots) of the strip's rows
      for (int q = p.slot_lo[si.strip_base + s]; q < si.slots; q += egroups) {
        auto it = written[s].find(q / egroups);
        if (it == written[s].end() || it->second != 1) fail("slot not written once", s, q);
      }
    }
    // band units: one per evaluated strip of the first series (the band seeds bounds)
    int nb = 0;
    for (int u = p.nunits; u < p.nunits + p.nband; ++u) {
      const WorkUnit& w = p.units[u];
      if (w.series != b) continue;
      ++nb;
      if (w.jlo < 0 || w.jhi > M || w.jlo >= w.jhi) fail("band columns", b, u);
      if (pstrip.empty() && (w.jlo > w.strip * R || w.jhi < std::min(M, w.strip * R + R)))
        fail("band misses the strip's block", b, w.strip);
    }
    if (nb != shi - slo) fail("band units per strip", nb, shi - slo);
  }
  // phases
  const int K = pstrip.empty() ? 1 : (int)pstrip.size() - 1;
  if ((int)p.pu.size() != K + 1 || p.pu[0] != 0 || p.pu[K] != p.nunits) fail("main phases", K, 0);
  if ((int)p.pb.size() != K + 1 || p.pb[0] != p.nunits || p.pb[K] != p.nunits + p.nband)
    fail("band phases", K, 0);
  if (!pstrip.empty()) {
    const int R = p.table.s[0].rows_out;
    if (pstrip[1] * R > mean_first((int)N0)) fail("phase 0 lacks the mean's days", pstrip[1], 0);
    for (int q = 0; q < K; ++q) {
      const int first_day = pstrip[q + 1] * R;
      for (int u = p.pu[q]; u < p.pu[q + 1]; ++u) {
        const WorkUnit& w = p.units[u];
        if (w.strip < pstrip[q + 1] || w.strip >= pstrip[q]) fail("unit in another phase", q, u);
        if (w.jlo < first_day) fail("unit reads days not yet copied", q, u);
      }
      for (int u = p.pb[q]; u < p.pb[q + 1]; ++u)
        if (p.units[u].jlo < first_day) fail("band unit reads days not yet copied", q, u);
    }
  }
}

void check_shape(int64_t N, int64_t D, int L, int emb, int sym, int want_tiles, int want_group,
                 int B = 1, int64_t N_last = 0) {
  traknn_ctx h;
  h.sm_count = 152;
  h.sym = sym;
  std::vector<HostSeries> sd(B);
  for (int b = 0; b < B; ++b) {  // B series, lengths spread evenly from N to N_last
    const int64_t Nb = B > 1 ? N + (N_last - N) * b / (B - 1) : N;
    sd[b] = HostSeries{nullptr, Nb, L, 20, L - 1, nullptr, nullptr, nullptr};
  }
  int tiles = 8, group = 0;
  default_shape(&h, sd.data(), B, D, emb, 0, INT_MAX, &tiles, &group);
  if (tiles != want_tiles || group != want_group) fail("default unit shape", tiles, group);
}

}  // namespace

int main() {
  for (int tiles : {2, 4, 8, 16}) {
    check_plan(1, 27394, 5, tiles, 19, 1, 1, 0, INT_MAX, {}, 2);
    check_plan(1, 27394, 1, tiles, 38, 2, 1, 0, INT_MAX, {}, 8);
  }
  check_plan(1, 27394, 17, 8, 19, 1, 1, 0, INT_MAX, {}, 2);
  check_plan(1, 5000, 5, 8, 19, 1, 0, 0, INT_MAX, {}, 2);   // both triangles
  check_plan(1, 5000, 3, 4, 7, 1, 1, 10, 25, {}, 2);        // one part of a split series
  check_plan(1, 5000, 3, 4, 7, 1, 1, 0, 9, {}, 2);
  check_plan(1, 300, 2, 8, 19, 1, 1, 0, INT_MAX, {}, 2);
  check_plan(1, 20, 2, 8, 19, 1, 1, 0, INT_MAX, {}, 2);     // one partial strip
  check_plan(5, 6000, 3, 4, 19, 1, 1, 0, INT_MAX, {}, 2);   // batched, uneven series
  // host-buffer calls in phases: long series are split; a series is not when it has
  // fewer than 8 strips or when phase 0 (which holds the last 4,096 days, read by the
  // centring mean) would take nearly all of it
  for (int64_t N : {300, 1000, 1100, 3000, 5000, 9000, 15000, 27394})
    for (int L : {2, 5, 17}) {
      const int R = kTileRows - (L - 1);
      const int strips = (int)((N - L + 1 + R - 1) / R);
      const std::vector<int> ps = phase_plan(strips, R, N);
      if ((strips < 8 || N <= kMeanDays) && !ps.empty()) fail("phase split", (int)N, L);
      if (N >= 9000 && ps.empty()) fail("long series not split", (int)N, L);
      if (!ps.empty()) {
        if (ps.front() != strips || ps.back() != 0) fail("phase ends", (int)N, L);
        for (size_t q = 0; q + 1 < ps.size(); ++q)
          if (ps[q + 1] >= ps[q]) fail("phase order", (int)N, L);
        for (int tiles : {2, 8}) check_plan(1, N, L, tiles, 19, 1, 1, 0, INT_MAX, ps, 2);
      }
    }
  // unit length: 8 tiles at the 75-year length, shorter for shorter series, 16 tiles
  // and 38 strips for short operand rows
  check_shape(27394, 3726, 5, 1, 1, 8, 0);
  check_shape(20546, 3726, 5, 1, 1, 4, 0);
  check_shape(13697, 3726, 5, 1, 1, 4, 0);
  check_shape(10957, 3726, 5, 1, 1, 2, 0);
  check_shape(10957, 3726, 5, 1, 0, 4, 0);  // both triangles: twice the tiles
  check_shape(27394, 32, 5, 5, 1, 16, 38);
  // long operand rows: at most 65,536 K entries x tiles per unit, two tiles at least
  check_shape(27394, 58101, 5, 1, 1, 2, 0);
  check_shape(27394, 12000, 5, 1, 1, 4, 0);
  check_shape(10957, 58101, 5, 1, 1, 2, 0);
  // several series: the average series decides
  check_shape(27394, 3726, 5, 1, 1, 8, 0, 4, 27394);
  check_shape(3650, 3726, 5, 1, 1, 4, 0, 64, 27394);
  check_shape(3650, 3726, 5, 1, 1, 2, 0, 8, 9000);
  std::printf("%s\n", g_fail ? "plan check failed" : "plan check ok");
  return g_fail ? 1 : 0;
}
