// Exhaustive host-side check of the pass routing (route_passes): for every
// pass count and every pattern of trivial (skipped) passes, in place and out
// of place, simulate which buffer holds which version of the data.  Built with
// nvcc and run on the host by tests/test_route_passes.py; launches nothing.
#include <cstdio>

#include "../paper_2605_10390_gb300/csrc/fsort_dev.cuh"

using namespace fsort;

int main() {
  long cases = 0, bad = 0;
  for (int passes = 0; passes <= kMaxPasses; ++passes) {
    for (long mask = 0; mask < (1L << passes); ++mask) {
      for (int in_place = 0; in_place < 2; ++in_place) {
        int trivial[kMaxPasses] = {};
        int k = 0;
        for (int j = 0; j < passes; ++j) {
          trivial[j] = int((mask >> j) & 1);
          k += trivial[j] ? 0 : 1;
        }
        Schedule s{};
        route_passes(trivial, passes, in_place, &s);
        // version[b]: how many passes the data in buffer b has been through
        // (-1: no data); the input holds version 0
        int version[3] = {0, -1, -1};
        int done = 0;
        bool ok = s.active_passes == k;
        for (int j = 0; j < kMaxPasses && ok; ++j) {
          const PassDesc& p = s.pass[j];
          const bool should = j < passes && !trivial[j];
          if (p.active != (should ? 1 : 0)) ok = false;
          if (!p.active) continue;
          if (p.src < 0 || p.src > 2 || p.dst < 0 || p.dst > 2 || p.src == p.dst) ok = false;
          else if (version[p.src] != done) ok = false;            // reads the latest data
          else if (!in_place && p.dst == kBufIn) ok = false;      // the input is read-only
          else version[p.dst] = ++done;
        }
        const int target = in_place ? kBufIn : kBufOut;
        if (ok) {
          const PassDesc& c = s.copy;
          int holder = -1;  // the buffer with the final version
          for (int b = 0; b < 3; ++b)
            if (version[b] == done) holder = b;
          if (c.active != (holder != target ? 1 : 0)) ok = false;   // a copy exactly when needed
          // and the routing needs one only when no assignment can avoid it: out of place when
          // every pass is skipped, in place after an odd number of passes
          if (c.active != (in_place ? (k & 1) : (k == 0))) ok = false;
          if (c.active && (c.src != holder || c.dst != target)) ok = false;
          if (c.active) version[target] = done;
          if (version[target] != k) ok = false;                    // every active pass, in order
        }
        ++cases;
        if (!ok) {
          if (++bad <= 10) std::printf("bad: passes %d mask %lx in_place %d\n", passes, mask, in_place);
        }
      }
    }
  }
  std::printf("cases %ld bad %ld\n", cases, bad);
  return bad ? 1 : 0;
}
